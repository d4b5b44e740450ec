// Explicit local interface operators (Sec. 3.2 applied once per subdomain instead of once
// per iteration): for every subdomain s, with b_s the local dofs touched by B_s,
//   F_s = (K_s^+)_{b_s b_s}                       (so F = sum_s B_s F_s B_s^T, Eq. 3.6),
//   S_s = K_bb - K_bi K_ii^{-1} K_ib               (the Dirichlet preconditioner, Eq. 3.5),
// both dense m_s x m_s, built at factorisation time by multi-right-hand-side solves with
// the band factors, and applied in the PCG loop as batched dense products.
//
// Build: one CTA per (subdomain, tile of MT = 32 right-hand sides), persistent over a work
// queue.  The tile's n x MT block lives in a per-CTA global scratch; the forward and
// backward sweeps keep the b + 32 live rows in a shared-memory window (cyclic in the row
// index), stage the 32 factor columns of the current block and its inverse diagonal block
// in shared memory, and do the off-block coupling as a register-tiled product (8 rows x 4
// columns per thread in the forward sweep, 1 row x 4 columns in the backward sweep).
// No spin-waits and no asynchronous copies: plain loads and __syncthreads only.
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "device.cuh"

namespace fp {

template <typename T>
__device__ __forceinline__ void ld4(const T *p, T (&v)[4]) {
  v[0] = p[0]; v[1] = p[1]; v[2] = p[2]; v[3] = p[3];
}

// Scalar arithmetic of the build, per element type.  float and double: plain FMAs (the same
// values as the contracted a += x * y).  dfl: a two-float value h + l (the FP64 factor split
// once, two_sum / TwoProduct by fma as in device.cuh), ~2^-46 relative per operation, which gives
// F_s to FP64-like accuracy from FP32 instructions: GB300 issues FP64 FMAs at about 1/60 of the FP32
// rate, and a two-float multiply-add costs 15 FP32 instructions.
struct __align__(8) dfl {
  float h, l;
};
template <typename T> __device__ __forceinline__ T num(double v);
template <> __device__ __forceinline__ float num<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ double num<double>(double v) { return v; }
template <> __device__ __forceinline__ dfl num<dfl>(double v) {
  dfl r;
  df_split(v, r.h, r.l);
  return r;
}
__device__ __forceinline__ double to_double(float v) { return v; }
__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ double to_double(dfl v) { return (double)v.h + (double)v.l; }
template <typename TO, typename T> __device__ __forceinline__ TO out_of(T v) { return v; }
template <> __device__ __forceinline__ double out_of<double, dfl>(dfl v) { return to_double(v); }
// Long sums: a += x * y with the two-float sum left unnormalised (the high part takes the exact
// TwoSum, the low part collects its error and the product's), so the loop-carried chain is one
// addition per part; norm() restores h + l with |l| <= ulp(h) / 2 before the value is used
// (TwoSum: after cancellation the low part can be the larger one).
// float and double: the plain FMA.
__device__ __forceinline__ void fma_lazy(float &a, float x, float y) { a = fmaf(x, y, a); }
__device__ __forceinline__ void fma_lazy(double &a, double x, double y) { a = fma(x, y, a); }
__device__ __forceinline__ void fma_lazy(dfl &a, dfl x, dfl y) {
  const float p = x.h * y.h;
  const float pe = fmaf(x.l, y.h, fmaf(x.h, y.l, fmaf(x.h, y.h, -p)));
  float s, e;
  two_sum(a.h, p, s, e);
  a.h = s;
  a.l += e + pe;
}
__device__ __forceinline__ void fms_lazy(float &a, float x, float y) { a = fmaf(-x, y, a); }
__device__ __forceinline__ void fms_lazy(double &a, double x, double y) { a = fma(-x, y, a); }
__device__ __forceinline__ void fms_lazy(dfl &a, dfl x, dfl y) { fma_lazy(a, dfl{-x.h, -x.l}, y); }
__device__ __forceinline__ void norm(float &) {}
__device__ __forceinline__ void norm(double &) {}
__device__ __forceinline__ void norm(dfl &a) { df_norm(a.h, a.l); }
// a -= b
__device__ __forceinline__ void sub_from(float &a, float b) { a -= b; }
__device__ __forceinline__ void sub_from(double &a, double b) { a -= b; }
__device__ __forceinline__ void sub_from(dfl &a, dfl b) { df_add(a.h, a.l, -b.h, -b.l); }
// x * y
__device__ __forceinline__ float mul(float x, float y) { return x * y; }
__device__ __forceinline__ double mul(double x, double y) { return x * y; }
__device__ __forceinline__ dfl mul(dfl x, dfl y) {
  dfl r;
  float hh, ll;
  df_mul(x.h, x.l, y.h, y.l, hh, ll);
  r.h = hh + ll;
  r.l = ll - (r.h - hh);
  return r;
}

// Copies ncb rows of LD elements (stride LD in global, LDp in shared memory; LD a multiple of 32,
// LDp of 4, so every row starts 16-byte aligned on both sides) with 16-byte loads, one warp per row.
template <typename T>
__device__ __forceinline__ void stage_rows(T *dst, int LDp, const T *src, int LD, int ncb) {
  constexpr int V = 16 / sizeof(T);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = warp; c < ncb; c += nw) {
    const uint4 *sp = reinterpret_cast<const uint4 *>(src + (long long)c * LD);
    uint4 *dp = reinterpret_cast<uint4 *>(dst + (size_t)c * LDp);
    for (int v = lane; v < LD / V; v += 32) dp[v] = sp[v];
  }
}

// kind 0: F_s (right-hand sides e_{b_j}; fixed dofs of floating subdomains give zero
// columns), kind 1: S_s (right-hand sides -K_{i, b_j} on interior rows, Dirichlet factor).
// Task t = (subdomain task_s[t], first column task_j0[t]); MT right-hand sides per task
// (32, or 16 where a 32-wide window does not fit in shared memory).  Thread layout: CG = MT/4
// column groups of 4, RG = 256/CG row groups; NR = ceil(b / RG) rows per thread in the
// forward coupling; only the first 32 row groups work on the 32-row diagonal blocks.
// T: the arithmetic and storage type of factor, inverse blocks, window and scratch (float, double,
// or dfl); TO: the operator's element type (T, or double for dfl).
template <typename T, typename TO, int NR, int MT>
__global__ void __launch_bounds__(256) k_band_mrhs(const int *task_s, const int *task_j0, int ntask, DevTopo D,
                                                   const T *fac, const T *linv, const long long *linv_off,
                                                   const double *csr_val, int kind, T *scratch,
                                                   long long scratch_stride, int *counter, TO *out,
                                                   const long long *out_off, int R, int LDp) {
  constexpr int CG = MT / 4, RG = 256 / CG;
  extern __shared__ __align__(16) unsigned char smraw[];
  T *Wn = reinterpret_cast<T *>(smraw);  // R x MT window
  T *Fc = Wn + (size_t)R * MT;           // 32 x LDp staged factor columns
  T *Lv = Fc + (size_t)32 * LDp;         // 32 x 32 inverse diagonal block
  T *Tt = Lv + 1024;                     // 32 x MT backward temporaries
  __shared__ int s_task;
  const int tid = threadIdx.x, cg = tid % CG, rg = tid / CG;
  T *Xs = scratch + (long long)blockIdx.x * scratch_stride;
  for (;;) {
    if (tid == 0) s_task = atomicAdd(counter, 1);
    __syncthreads();
    const int task = s_task;
    __syncthreads();
    if (task >= ntask) break;
    const int s = task_s[task], j0 = task_j0[task];
    const DevTpl t = D.tpl[D.sub_tpl[s]];
    const int n = t.n, LD = t.LD, b = t.b, m = t.nbnd;
    const int ncol = min(MT, m - j0);
    const int *bnd = D.pool + t.bnd;
    const int *cptr = D.pool + t.csr_ptr, *ccol = D.pool + t.csr_col;
    const int *isb = D.pool + t.is_bnd;
    const double *val = csr_val + D.csr_off[s];
    const T *F = fac + D.fac_off[s];
    const T *Li = linv + linv_off[s];
    auto fixed = [&](int d) { return t.floating && (d == t.fixed0 || d == t.fixed1 || d == t.fixed2); };
    // ---- right-hand sides into the scratch block (row r at Xs + r * MT) ----
    for (long long i = tid; i < (long long)n * MT; i += blockDim.x) Xs[i] = num<T>(0.0);
    __syncthreads();
    for (int jj = tid; jj < ncol; jj += blockDim.x) {
      const int c = bnd[j0 + jj];
      if (kind == 0) {
        if (!fixed(c)) Xs[(long long)c * MT + jj] = num<T>(1.0);
      } else {
        for (int e = cptr[c]; e < cptr[c + 1]; ++e) {
          const int i = ccol[e];
          if (!isb[i]) Xs[(long long)i * MT + jj] = num<T>(-val[e]);
        }
      }
    }
    __syncthreads();
    const int nb = (n + 31) / 32;
    // The tile's right-hand sides vanish above row rs (kind 0: the unit vectors start at b_j0,
    // the smallest of the tile's dofs, b sorted; kind 1: K's band reaches b_j0 - b), so the
    // forward sweep starts at block k0.  Only the operator's entries (a, j) with a >= j0 are
    // formed (the rest by symmetry, k_mrhs_symmetrize): they need the solution at rows >= b_j0
    // (kind 0) or >= b_j0 - b (kind 1), so the backward sweep stops at the same block k0.
    const int rs = kind == 0 ? bnd[j0] : max(0, bnd[j0] - b);
    const int k0 = rs / 32;
    // ---- forward sweep: L y = rhs, z = D^{-1} y into Xs ----
    int hi = 32 * k0;
    for (int k = k0; k < nb; ++k) {
      const int r0 = 32 * k, ncb = min(32, n - r0), rend = min(n, r0 + 32 + b);
      for (int idx = tid; idx < (rend - hi) * MT; idx += blockDim.x) {
        const int r = hi + idx / MT, q = idx % MT;
        Wn[(r % R) * MT + q] = Xs[(long long)r * MT + q];
      }
      hi = max(hi, rend);
      stage_rows(Fc, LDp, F + (long long)r0 * LD, LD, ncb);
      stage_rows(Lv, 32, Li + (long long)k * 1024, 32, 32);
      __syncthreads();
      const int rw0 = r0 % R;  // window slot of row r0 (rows r0 .. r0 + 31 never wrap past R twice)
      // diagonal block: y_k = Linv_k w_k (rows past n are never loaded: c < ncb)
      T y[4] = {num<T>(0.0), num<T>(0.0), num<T>(0.0), num<T>(0.0)};
      if (rg < 32) {
        for (int c = 0; c < ncb; ++c) {
          const T l = Lv[rg * 32 + c];
          T w[4];
          const int rw = rw0 + c < R ? rw0 + c : rw0 + c - R;
          ld4(Wn + rw * MT + 4 * cg, w);
#pragma unroll
          for (int q = 0; q < 4; ++q) fma_lazy(y[q], l, w[q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) norm(y[q]);
      }
      __syncthreads();
      if (rg < ncb) {
        const T dinv = Fc[rg * LDp + (r0 + rg) % LD];
        T *wr = Wn + ((r0 + rg) % R) * MT + 4 * cg;
        T *xr = Xs + (long long)(r0 + rg) * MT + 4 * cg;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          wr[q] = y[q];
          xr[q] = mul(y[q], dinv);
        }
      }
      __syncthreads();
      // off-block coupling: w_r -= sum_c L(r, r0 + c) y_{r0 + c}, r in [r0 + 32, rend)
      T acc[NR][4];
#pragma unroll
      for (int i = 0; i < NR; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] = num<T>(0.0);
      int sl[NR];  // slot of row r0 + 32 + rg + RG i in a factor column
#pragma unroll
      for (int i = 0; i < NR; ++i) sl[i] = (r0 + 32 + rg + RG * i) % LD;
      for (int c = 0; c < ncb; ++c) {
        T yc[4];
        const int rw = rw0 + c < R ? rw0 + c : rw0 + c - R;
        ld4(Wn + rw * MT + 4 * cg, yc);
        const T *col = Fc + c * LDp;
#pragma unroll
        for (int i = 0; i < NR; ++i) {
          const int r = r0 + 32 + rg + RG * i;
          const T l = (r < rend && r - (r0 + c) <= b) ? col[sl[i]] : num<T>(0.0);
#pragma unroll
          for (int q = 0; q < 4; ++q) fma_lazy(acc[i][q], l, yc[q]);
        }
      }
#pragma unroll
      for (int i = 0; i < NR; ++i) {
        const int r = r0 + 32 + rg + RG * i;
        if (r < rend) {
#pragma unroll
          for (int q = 0; q < 4; ++q) norm(acc[i][q]);
          T *wr = Wn + (r % R) * MT + 4 * cg;
#pragma unroll
          for (int q = 0; q < 4; ++q) sub_from(wr[q], acc[i][q]);
        }
      }
      __syncthreads();
    }
    // ---- backward sweep: L^T x = z; x rows kept in the window and written to Xs ----
    for (int k = nb - 1; k >= k0; --k) {
      const int r0 = 32 * k, ncb = min(32, n - r0), rtop = min(n, r0 + 32 + b);
      stage_rows(Fc, LDp, F + (long long)r0 * LD, LD, ncb);
      stage_rows(Lv, 32, Li + (long long)k * 1024, 32, 32);
      __syncthreads();
      T tv[4] = {num<T>(0.0), num<T>(0.0), num<T>(0.0), num<T>(0.0)};
      if (rg < ncb) {
        ld4(Xs + (long long)(r0 + rg) * MT + 4 * cg, tv);
        const T *col = Fc + rg * LDp;
        const int j = r0 + rg;
        // slots of row r in a factor column (mod LD) and in the window (mod R), stepped with r
        int rl = (r0 + 32) % LD, rw = (r0 + 32) % R;
        for (int r = r0 + 32; r < rtop; ++r) {
          const T l = (r - j <= b) ? col[rl] : num<T>(0.0);
          T x4[4];
          ld4(Wn + rw * MT + 4 * cg, x4);
#pragma unroll
          for (int q = 0; q < 4; ++q) fms_lazy(tv[q], l, x4[q]);
          if (++rl == LD) rl = 0;
          if (++rw == R) rw = 0;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) norm(tv[q]);
      }
      if (rg < 32) {
#pragma unroll
        for (int q = 0; q < 4; ++q) Tt[rg * MT + 4 * cg + q] = tv[q];
      }
      __syncthreads();
      // within the block: x_k = Linv_k^T t
      T x[4] = {num<T>(0.0), num<T>(0.0), num<T>(0.0), num<T>(0.0)};
      if (rg < 32) {
#pragma unroll 8
        for (int c = 0; c < 32; ++c) {
          const T l = Lv[c * 32 + rg];
          T tc[4];
          ld4(Tt + c * MT + 4 * cg, tc);
#pragma unroll
          for (int q = 0; q < 4; ++q) fma_lazy(x[q], l, tc[q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) norm(x[q]);
      }
      if (rg < ncb) {
        T *wr = Wn + ((r0 + rg) % R) * MT + 4 * cg;
        T *xr = Xs + (long long)(r0 + rg) * MT + 4 * cg;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          wr[q] = x[q];
          xr[q] = x[q];
        }
      }
      __syncthreads();
    }
    // ---- the operator's columns j0 .. j0 + ncol - 1 ----
    TO *O = out + out_off[s];
    const int mp = (m + 3) & ~3;  // row stride (padded to 4 for vector loads)
    const int mlow = m - j0;  // rows a = j0 .. m - 1
    if (kind == 0) {
      for (int idx = tid; idx < mlow * ncol; idx += blockDim.x) {
        const int a = j0 + idx / ncol, jj = idx % ncol;
        O[(long long)a * mp + j0 + jj] = out_of<TO>(Xs[(long long)bnd[a] * MT + jj]);
      }
    } else {
      // S[a][j] = sum_c K[b_a][c] (y_j[c] + [c == b_j]);  y_j vanishes on the rows of b
      for (int idx = tid; idx < mlow * ncol; idx += blockDim.x) {
        const int a = j0 + idx / ncol, jj = idx % ncol;
        const int row = bnd[a], cj = bnd[j0 + jj];
        double acc = 0.0;
        for (int e = cptr[row]; e < cptr[row + 1]; ++e) {
          const int c = ccol[e];
          acc += val[e] * (to_double(Xs[(long long)c * MT + jj]) + (c == cj ? 1.0 : 0.0));
        }
        O[(long long)a * mp + j0 + jj] = TO(acc);
      }
    }
    __syncthreads();
  }
}

// Completes an operator built by k_band_mrhs (entries (a, j) formed for a >= the first column
// of j's tile of MT right-hand sides): A[a][j] = A[j][a] for the rest.  One CTA per subdomain.
template <typename T>
__global__ void k_mrhs_symmetrize(DevTopo D, T *out, const long long *out_off, int MT) {
  const int s = blockIdx.x;
  const DevTpl t = D.tpl[D.sub_tpl[s]];
  const int m = t.nbnd, mp = (m + 3) & ~3;
  T *O = out + out_off[s];
  for (long long idx = threadIdx.x; idx < (long long)m * m; idx += blockDim.x) {
    const int a = (int)(idx / m), j = (int)(idx % m);
    if (a < (j / MT) * MT) O[(long long)a * mp + j] = O[(long long)j * mp + a];
  }
}

// y_b = A_s x_b for every subdomain (A_s = F_s or S_s, dense, row stride mp = m rounded up
// to 4, pad columns zero), read from and written back to the local vectors at the rows b_s
// (in place: x_b is staged in shared memory first).  One CTA per subdomain; a warp takes four
// rows at a time (vectorised row loads, x read once for the four), accumulates each with plain
// FMAs and reduces the four lane sums together: two transposing exchanges (offsets 16, 8) leave
// one row per lane octet, three more steps finish it: 6 additions per lane for four rows
// instead of 5 per row.  Sums in the operator's precision.
template <typename T>
__global__ void __launch_bounds__(256) k_explicit_apply(DevTopo D, const T *ops, const long long *op_off,
                                                        double *xloc, const int *fl) {
  if (fl && fl[FL_DONE]) return;
  extern __shared__ unsigned char smraw[];
  T *xs = reinterpret_cast<T *>(smraw);
  const int s = blockIdx.x;
  const DevTpl t = D.tpl[D.sub_tpl[s]];
  const int m = t.nbnd, mp = (m + 3) & ~3;
  const int *bnd = D.pool + t.bnd;
  double *x = xloc + D.vec_off[s];
  for (int q = threadIdx.x; q < mp; q += blockDim.x) xs[q] = q < m ? T(x[bnd[q]]) : T(0);
  __syncthreads();
  const T *A = ops + op_off[s];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int a0 = 4 * warp; a0 < m; a0 += 4 * nw) {
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (int j = 4 * lane; j < mp; j += 128) {
      const T x0 = xs[j], x1 = xs[j + 1], x2 = xs[j + 2], x3 = xs[j + 3];
#pragma unroll
      for (int rr = 0; rr < 4; ++rr) {
        if (a0 + rr < m) {
          const T *row = A + (long long)(a0 + rr) * mp;
          T v[4];
          if (sizeof(T) == 4) {
            const float4 f = *reinterpret_cast<const float4 *>(row + j);
            v[0] = T(f.x); v[1] = T(f.y); v[2] = T(f.z); v[3] = T(f.w);
          } else {
            const double2 d0 = *reinterpret_cast<const double2 *>(row + j);
            const double2 d1 = *reinterpret_cast<const double2 *>(row + j + 2);
            v[0] = T(d0.x); v[1] = T(d0.y); v[2] = T(d1.x); v[3] = T(d1.y);
          }
          acc[rr] = fma(v[0], x0, acc[rr]);
          acc[rr] = fma(v[1], x1, acc[rr]);
          acc[rr] = fma(v[2], x2, acc[rr]);
          acc[rr] = fma(v[3], x3, acc[rr]);
        }
      }
    }
    // lanes with bit 4 set keep rows 2, 3, the others rows 0, 1; then bit 3 picks one of the two
    const bool hi16 = (lane & 16) != 0, hi8 = (lane & 8) != 0;
    T k0 = hi16 ? acc[2] : acc[0], k1 = hi16 ? acc[3] : acc[1];
    k0 += __shfl_xor_sync(FULL, hi16 ? acc[0] : acc[2], 16);
    k1 += __shfl_xor_sync(FULL, hi16 ? acc[1] : acc[3], 16);
    T k = hi8 ? k1 : k0;
    k += __shfl_xor_sync(FULL, hi8 ? k0 : k1, 8);
    k += __shfl_xor_sync(FULL, k, 4);
    k += __shfl_xor_sync(FULL, k, 2);
    k += __shfl_xor_sync(FULL, k, 1);
    const int a = a0 + 2 * (hi16 ? 1 : 0) + (hi8 ? 1 : 0);
    if ((lane & 7) == 0 && a < m) x[bnd[a]] = double(k);
  }
}

// ---------------------------- symmetric tiled FP32 operators ----------------------------
// The PCG loop's FP32 operators are stored as the upper 32 x 32 tiles (I <= J) of A_s, tile
// index I nt - I (I - 1) / 2 + (J - I) with nt = ceil(m / 32), row-major inside a tile and
// zero past m: about half the bytes of the full matrix, and exactly symmetric.
__device__ __forceinline__ void tile_ij(int tile, int nt, int &I, int &J) {
  I = 0;
  while (tile >= nt - I) {
    tile -= nt - I;
    ++I;
  }
  J = I + tile;
}

__device__ __forceinline__ void store_tile_elem(float *p, float v) { *p = v; }
__device__ __forceinline__ void store_tile_elem(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ float load_tile_elem(const float *p) { return *p; }
__device__ __forceinline__ float load_tile_elem(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
// two adjacent elements (p even-aligned)
__device__ __forceinline__ void load_tile_pair(const float *p, float &a, float &b) {
  const float2 v = *reinterpret_cast<const float2 *>(p);
  a = v.x;
  b = v.y;
}
__device__ __forceinline__ void load_tile_pair(const __nv_bfloat16 *p, float &a, float &b) {
  const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
  a = v.x;
  b = v.y;
}

template <typename Tin, typename Tout>
__global__ void k_pack_sym(DevTopo D, const Tin *full, const long long *full_off, Tout *tiles,
                           const long long *tile_off) {
  const int s = blockIdx.x;
  const DevTpl t = D.tpl[D.sub_tpl[s]];
  const int m = t.nbnd, mp = (m + 3) & ~3, nt = (m + 31) / 32, ntile = nt * (nt + 1) / 2;
  const Tin *Fm = full + full_off[s];
  Tout *Tm = tiles + tile_off[s];
  for (long long idx = threadIdx.x; idx < (long long)ntile * 1024; idx += blockDim.x) {
    int I, J;
    tile_ij((int)(idx >> 10), nt, I, J);
    const int e = (int)(idx & 1023), a = 32 * I + (e >> 5), j = 32 * J + (e & 31);
    store_tile_elem(Tm + idx, (a < m && j < m) ? float(Fm[(long long)a * mp + j]) : 0.0f);
  }
}

// y_b = A_s x_b for the tiled symmetric A_s, in place on the local vectors at the rows b_s.
// Warp w takes tiles w, w + 8, ...; a lane holds a pair of adjacent columns of every other row
// (16 loads of two whole rows per warp and tile).  An off-diagonal tile gives A_IJ^T x_I to y_J
// (per-lane column sums, the two row parities added across the half-warps) and A_IJ x_J to y_I:
// the 32 row sums come out of a transposing butterfly within each half-warp (at offset k a lane
// keeps the half of its values selected by bit k of its column-pair index and adds the
// partner's copy of that half: 15 shuffles).  Partial sums land in shared memory and are added
// in a fixed order.
// With vlam given, x_b is formed here from the multiplier vector (x_b = B_s^T vlam, the fixed
// dofs of a floating subdomain zero when skip_fixed), as k_scatter would, instead of being read
// from the local vector: one launch and one pass over the rows b_s fewer per apply.
// TS: the tiles' storage type (FP32, or BF16 for the preconditioner's S_s: half the bytes; the
// products and sums stay FP32).
template <typename TS>
__global__ void __launch_bounds__(256) k_explicit_apply_sym(DevTopo D, const TS *tiles, const long long *tile_off,
                                                            double *xloc, const int *fl, const double *vlam,
                                                            int skip_fixed) {
  if (fl && fl[FL_DONE]) return;
  extern __shared__ float smf[];
  const int s = blockIdx.x;
  const DevTpl t = D.tpl[D.sub_tpl[s]];
  const int m = t.nbnd, nt = (m + 31) / 32, ntile = nt * (nt + 1) / 2;
  float *xs = smf;                 // nt * 32
  float *rp = xs + nt * 32;        // ntile * 32 row-part sums
  float *cp = rp + ntile * 32;     // ntile * 32 column-part sums
  const int *bnd = D.pool + t.bnd;
  double *x = xloc + D.vec_off[s];
  if (vlam) {
    const long long b0 = D.bsc_off[s];
    for (int q = threadIdx.x; q < nt * 32; q += blockDim.x) {
      double acc = 0.0;
      if (q < m) {
        const int d = bnd[q];
        if (!(skip_fixed && t.floating && (d == t.fixed0 || d == t.fixed1 || d == t.fixed2))) {
#pragma unroll
          for (int z = 0; z < 3; ++z) {
            const int r = D.bsc_row[3 * (b0 + q) + z];
            if (r >= 0) acc += D.bsc_sign[3 * (b0 + q) + z] * vlam[r];
          }
        }
      }
      xs[q] = float(acc);
    }
  } else {
    for (int q = threadIdx.x; q < nt * 32; q += blockDim.x) xs[q] = q < m ? float(x[bnd[q]]) : 0.0f;
  }
  __syncthreads();
  const TS *A = tiles + tile_off[s];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // lane (h, c) = (lane >> 4, lane & 15) holds columns 2c, 2c + 1 of the rows 2i + h (i < 16): one
  // load instruction brings two whole rows (coalesced), 16 per tile
  const int h = lane >> 4, c = lane & 15;
  for (int tile = warp; tile < ntile; tile += nw) {
    int I, J;
    tile_ij(tile, nt, I, J);
    const TS *T = A + (long long)tile * 1024;
    float v0[16], v1[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) load_tile_pair(T + (2 * i + h) * 32 + 2 * c, v0[i], v1[i]);
    if (I < J) {  // A_IJ^T x_I: column sums, the two row parities added across the half-warps
      float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const float xr = xs[32 * I + 2 * i + h];
        a0 += v0[i] * xr;
        a1 += v1[i] * xr;
      }
      a0 += __shfl_xor_sync(FULL, a0, 16);
      a1 += __shfl_xor_sync(FULL, a1, 16);
      if (h == 0) {
        cp[tile * 32 + 2 * c] = a0;
        cp[tile * 32 + 2 * c + 1] = a1;
      }
    }
    // A_IJ x_J: the lane's part of row 2i + h, then a transposing butterfly over the 16 lanes of
    // the half-warp (offsets 8, 4, 2, 1): lane (h, c) ends with the sum of row 2c + h
    const float xj0 = xs[32 * J + 2 * c], xj1 = xs[32 * J + 2 * c + 1];
#pragma unroll
    for (int i = 0; i < 16; ++i) v0[i] = v0[i] * xj0 + v1[i] * xj1;
#pragma unroll
    for (int k = 8; k >= 1; k >>= 1) {
      const bool up = (c & k) != 0;
#pragma unroll
      for (int i = 0; i < k; ++i) {
        const float send = up ? v0[i] : v0[i + k];
        const float keep = up ? v0[i + k] : v0[i];
        v0[i] = keep + __shfl_xor_sync(FULL, send, k);
      }
    }
    rp[tile * 32 + 2 * c + h] = v0[0];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const int I = i >> 5, r = i & 31;
    const int row0 = I * nt - I * (I - 1) / 2;  // tile index of (I, I)
    float y = 0.0f;
    for (int J = I; J < nt; ++J) y += rp[(row0 + J - I) * 32 + r];
    for (int I2 = 0; I2 < I; ++I2) y += cp[(I2 * nt - I2 * (I2 - 1) / 2 + I - I2) * 32 + r];
    x[bnd[i]] = double(y);
  }
}

// ------------------------- symmetric tiled two-float operators -------------------------
// The accurate applies of the mixed-precision path (reference, initial, learned-guess and true
// residuals) need F_s to FP64 accuracy.  F_s (formed in FP64) is kept as hi/lo FP32 pairs of its
// upper 32 x 32 tiles (hi = fl32(a), lo = fl32(a - hi); 2048 floats per tile at 2 x the tile
// offsets of the FP32 loop operator): the bytes of half the FP64 matrix, and FP32 arithmetic with
// error-free products and sums (two-float; ~1e-14 relative) instead of FP64 FMAs, which bound the
// FP64 apply on GB300.
__global__ void k_pack_sym2f(DevTopo D, const double *full, const long long *full_off, float *tiles,
                             const long long *tile_off) {
  const int s = blockIdx.x;
  const DevTpl t = D.tpl[D.sub_tpl[s]];
  const int m = t.nbnd, mp = (m + 3) & ~3, nt = (m + 31) / 32, ntile = nt * (nt + 1) / 2;
  const double *Fm = full + full_off[s];
  float *Tm = tiles + 2 * tile_off[s];
  for (long long idx = threadIdx.x; idx < (long long)ntile * 1024; idx += blockDim.x) {
    int I, J;
    const int tile = (int)(idx >> 10);
    tile_ij(tile, nt, I, J);
    const int e = (int)(idx & 1023), a = 32 * I + (e >> 5), j = 32 * J + (e & 31);
    const double v = (a < m && j < m) ? Fm[(long long)a * mp + j] : 0.0;
    float h, l;
    df_split(v, h, l);
    Tm[(long long)tile * 2048 + e] = h;
    Tm[(long long)tile * 2048 + 1024 + e] = l;
  }
}

// y_b = A_s x_b in two-float arithmetic, in place on the local vectors at the rows b_s: the
// tile schedule of k_explicit_apply_sym (a warp per tile, lane c holding column c; transposed
// product as a per-lane sum, direct product through the transposing butterfly), two-float
// partials in shared memory added in a fixed order; one rounding to FP64 per row.
__global__ void __launch_bounds__(256, 2) k_explicit_apply_sym2f(DevTopo D, const float *tiles,
                                                                 const long long *tile_off, double *xloc,
                                                                 const int *fl) {
  if (fl && fl[FL_DONE]) return;
  extern __shared__ float2 smd2[];
  const int s = blockIdx.x;
  const DevTpl t = D.tpl[D.sub_tpl[s]];
  const int m = t.nbnd, nt = (m + 31) / 32, ntile = nt * (nt + 1) / 2;
  float2 *rp = smd2;                 // ntile * 32 row-part sums (two-float)
  float2 *cp = rp + ntile * 32;      // ntile * 32 column-part sums
  float *xh = reinterpret_cast<float *>(cp + ntile * 32);  // nt * 32
  float *xl = xh + nt * 32;
  const int *bnd = D.pool + t.bnd;
  double *x = xloc + D.vec_off[s];
  for (int q = threadIdx.x; q < nt * 32; q += blockDim.x) {
    float h = 0.0f, l = 0.0f;
    if (q < m) df_split(x[bnd[q]], h, l);
    xh[q] = h;
    xl[q] = l;
  }
  __syncthreads();
  const float *A = tiles + 2 * tile_off[s];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int tile = warp; tile < ntile; tile += nw) {
    int I, J;
    tile_ij(tile, nt, I, J);
    const float *T = A + (long long)tile * 2048;
    float vh[32], vl[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      vh[r] = T[r * 32 + lane];
      vl[r] = T[1024 + r * 32 + lane];
    }
    if (I < J) {
      float sh = 0.0f, sl = 0.0f;
#pragma unroll
      for (int r = 0; r < 32; ++r) {
        float ph, pl;
        df_mul(vh[r], vl[r], xh[32 * I + r], xl[32 * I + r], ph, pl);
        df_add_lazy(sh, sl, ph, pl);
      }
      df_norm(sh, sl);
      cp[tile * 32 + lane] = make_float2(sh, sl);
    }
    const float yh = xh[32 * J + lane], yl = xl[32 * J + lane];
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      float ph, pl;
      df_mul(vh[r], vl[r], yh, yl, ph, pl);
      vh[r] = ph;
      vl[r] = pl;
    }
#pragma unroll
    for (int k = 16; k >= 1; k >>= 1) {
      const bool up = (lane & k) != 0;
#pragma unroll
      for (int i = 0; i < k; ++i) {
        const float sendh = up ? vh[i] : vh[i + k], sendl = up ? vl[i] : vl[i + k];
        float kh = up ? vh[i + k] : vh[i], kl = up ? vl[i + k] : vl[i];
        const float rh = __shfl_xor_sync(FULL, sendh, k), rl = __shfl_xor_sync(FULL, sendl, k);
        df_add_lazy(kh, kl, rh, rl);
        vh[i] = kh;
        vl[i] = kl;
      }
    }
    df_norm(vh[0], vl[0]);
    rp[tile * 32 + lane] = make_float2(vh[0], vl[0]);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const int I = i >> 5, r = i & 31;
    const int row0 = I * nt - I * (I - 1) / 2;
    float yh = 0.0f, yl = 0.0f;
    for (int J = I; J < nt; ++J) {
      const float2 q = rp[(row0 + J - I) * 32 + r];
      df_add_lazy(yh, yl, q.x, q.y);
    }
    for (int I2 = 0; I2 < I; ++I2) {
      const float2 q = cp[(I2 * nt - I2 * (I2 - 1) / 2 + I - I2) * 32 + r];
      df_add_lazy(yh, yl, q.x, q.y);
    }
    x[bnd[i]] = (double)yh + (double)yl;
  }
}

cudaError_t launch_pack_sym2f(DevTopo D, int S, const double *full, const long long *full_off, float *tiles,
                              const long long *tile_off, cudaStream_t st) {
  k_pack_sym2f<<<S, 256, 0, st>>>(D, full, full_off, tiles, tile_off);
  return cudaGetLastError();
}

cudaError_t launch_explicit_apply_sym2f(DevTopo D, int S, int mmax_bnd, const float *tiles, const long long *tile_off,
                                        double *xloc, const int *fl, cudaStream_t st) {
  const int nt = (mmax_bnd + 31) / 32;
  const size_t smem = sizeof(float2) * (size_t)nt * (nt + 1) * 32 + sizeof(float) * 2 * (size_t)nt * 32;
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(k_explicit_apply_sym2f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_explicit_apply_sym2f<<<S, 256, smem, st>>>(D, tiles, tile_off, xloc, fl);
  return cudaGetLastError();
}

// bf16_out: tiles are BF16 (tiles points to tile_total BF16 values), else FP32
cudaError_t launch_pack_sym(bool src_fp64, DevTopo D, int S, const void *full, const long long *full_off,
                            void *tiles, const long long *tile_off, cudaStream_t st, bool bf16_out) {
  if (bf16_out) {
    __nv_bfloat16 *tb = (__nv_bfloat16 *)tiles;
    if (src_fp64) k_pack_sym<double><<<S, 256, 0, st>>>(D, (const double *)full, full_off, tb, tile_off);
    else k_pack_sym<float><<<S, 256, 0, st>>>(D, (const float *)full, full_off, tb, tile_off);
  } else {
    float *tf = (float *)tiles;
    if (src_fp64) k_pack_sym<double><<<S, 256, 0, st>>>(D, (const double *)full, full_off, tf, tile_off);
    else k_pack_sym<float><<<S, 256, 0, st>>>(D, (const float *)full, full_off, tf, tile_off);
  }
  return cudaGetLastError();
}

cudaError_t launch_explicit_apply_sym(DevTopo D, int S, int mmax_bnd, const void *tiles, const long long *tile_off,
                                      double *xloc, const int *fl, cudaStream_t st, const double *vlam,
                                      int skip_fixed, bool bf16) {
  const int nt = (mmax_bnd + 31) / 32;
  const size_t smem = sizeof(float) * ((size_t)nt * 32 + (size_t)nt * (nt + 1) * 32);
  if (bf16) {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k_explicit_apply_sym<__nv_bfloat16>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    k_explicit_apply_sym<__nv_bfloat16><<<S, 256, smem, st>>>(D, (const __nv_bfloat16 *)tiles, tile_off, xloc, fl,
                                                              vlam, skip_fixed);
  } else {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k_explicit_apply_sym<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
      if (e != cudaSuccess) return e;
    }
    k_explicit_apply_sym<float><<<S, 256, smem, st>>>(D, (const float *)tiles, tile_off, xloc, fl, vlam, skip_fixed);
  }
  return cudaGetLastError();
}

// ------------------------------------ launchers --------------------------------------
template <typename T, typename TO, int NR, int MT>
static cudaError_t launch_mrhs_T(int grid, cudaStream_t st, const int *ts, const int *tj, int ntask, DevTopo D,
                                 const T *fac, const T *linv, const long long *loff, const double *csr, int kind,
                                 T *scratch, long long sstride, int *counter, TO *out, const long long *ooff, int R,
                                 int LDp, size_t smem) {
  cudaError_t e =
      cudaFuncSetAttribute(k_band_mrhs<T, TO, NR, MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_band_mrhs<T, TO, NR, MT><<<grid, 256, smem, st>>>(ts, tj, ntask, D, fac, linv, loff, csr, kind, scratch,
                                                      sstride, counter, out, ooff, R, LDp);
  return cudaGetLastError();
}

cudaError_t launch_mrhs_symmetrize(bool fp32, DevTopo D, int S, void *out, const long long *out_off, int mt,
                                   cudaStream_t st) {
  if (fp32) k_mrhs_symmetrize<float><<<S, 256, 0, st>>>(D, (float *)out, out_off, mt);
  else k_mrhs_symmetrize<double><<<S, 256, 0, st>>>(D, (double *)out, out_off, mt);
  return cudaGetLastError();
}

// prec: MRHS_FP64, MRHS_FP32 or MRHS_DF (two-float arithmetic, FP64 operator)
size_t mrhs_smem_bytes(int prec, int R, int LDp, int mt) {
  const size_t esz = prec == MRHS_FP32 ? 4 : 8;
  return esz * ((size_t)R * mt + 32 * (size_t)LDp + 1024 + 32 * (size_t)mt);
}

// rows per thread of the forward coupling for half bandwidth b: ceil(b / RG), RG = 256 / (MT / 4)
int mrhs_nr(int b, int mt) {
  const int rg = 256 / (mt / 4);
  const int nr = (b + rg - 1) / rg;
  return nr <= 4 ? 4 : nr <= 8 ? 8 : nr <= 12 ? 12 : nr <= 16 ? 16 : 0;
}

template <typename T, typename TO, int MT>
static const void *mrhs_fn(int nr) {
  return nr == 4 ? (const void *)k_band_mrhs<T, TO, 4, MT> : nr == 8 ? (const void *)k_band_mrhs<T, TO, 8, MT>
         : nr == 12 ? (const void *)k_band_mrhs<T, TO, 12, MT> : (const void *)k_band_mrhs<T, TO, 16, MT>;
}

cudaError_t launch_band_mrhs(int prec, int bmax, int mt, int grid, cudaStream_t st, const int *task_s,
                             const int *task_j0, int ntask, DevTopo D, const void *fac, const void *linv,
                             const long long *linv_off, const double *csr, int kind, void *scratch, long long sstride,
                             int *counter, void *out, const long long *out_off, int R, int LDp) {
  const size_t smem = mrhs_smem_bytes(prec, R, LDp, mt);
  const int nr = mrhs_nr(bmax, mt);
  if (nr == 0 || (mt != 32 && mt != 16)) return cudaErrorInvalidValue;
#define FP_MRHS(TT, TTO, N, M)                                                                                    \
  return launch_mrhs_T<TT, TTO, N, M>(grid, st, task_s, task_j0, ntask, D, (const TT *)fac, (const TT *)linv,     \
                                      linv_off, csr, kind, (TT *)scratch, sstride, counter, (TTO *)out, out_off, R, \
                                      LDp, smem)
#define FP_MRHS_NR(TT, TTO, M)            \
  if (nr == 4) FP_MRHS(TT, TTO, 4, M);    \
  if (nr == 8) FP_MRHS(TT, TTO, 8, M);    \
  if (nr == 12) FP_MRHS(TT, TTO, 12, M);  \
  FP_MRHS(TT, TTO, 16, M)
  if (prec == MRHS_FP32) {
    if (mt == 32) { FP_MRHS_NR(float, float, 32); }
    FP_MRHS_NR(float, float, 16);
  }
  if (prec == MRHS_DF) {
    if (mt == 32) { FP_MRHS_NR(dfl, double, 32); }
    FP_MRHS_NR(dfl, double, 16);
  }
  if (mt == 32) { FP_MRHS_NR(double, double, 32); }
  FP_MRHS_NR(double, double, 16);
#undef FP_MRHS_NR
#undef FP_MRHS
}

// resident CTAs per SM of the build kernel at this shared-memory size (0: does not fit)
int mrhs_blocks_per_sm(int prec, int bmax, int mt, int R, int LDp) {
  const size_t smem = mrhs_smem_bytes(prec, R, LDp, mt);
  const int nr = mrhs_nr(bmax, mt);
  if (nr == 0 || smem > 227 * 1024) return 0;
  const void *f = prec == MRHS_FP32 ? (mt == 32 ? mrhs_fn<float, float, 32>(nr) : mrhs_fn<float, float, 16>(nr))
                  : prec == MRHS_DF ? (mt == 32 ? mrhs_fn<dfl, double, 32>(nr) : mrhs_fn<dfl, double, 16>(nr))
                                    : (mt == 32 ? mrhs_fn<double, double, 32>(nr) : mrhs_fn<double, double, 16>(nr));
  if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, 256, smem) != cudaSuccess) return 0;
  return nb;
}

// Splits n FP64 values in place into two-float values (h, l) occupying the same 8 bytes.
__global__ void k_split_df(double *v, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    dfl r;
    df_split(v[i], r.h, r.l);
    reinterpret_cast<dfl *>(v)[i] = r;
  }
}

cudaError_t launch_split_df(double *v, long long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_split_df<<<1216, 256, 0, st>>>(v, n);
  return cudaGetLastError();
}

cudaError_t launch_explicit_apply(bool fp32, DevTopo D, int S, int mmax_bnd, const void *ops, const long long *op_off,
                                  double *xloc, const int *fl, cudaStream_t st) {
  const size_t smem = (size_t)((mmax_bnd + 3) & ~3) * (fp32 ? 4 : 8);
  if (fp32) k_explicit_apply<float><<<S, 256, smem, st>>>(D, (const float *)ops, op_off, xloc, fl);
  else k_explicit_apply<double><<<S, 256, smem, st>>>(D, (const double *)ops, op_off, xloc, fl);
  return cudaGetLastError();
}

}  // namespace fp
