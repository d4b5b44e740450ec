// Assembly of the local 3-field systems, load vectors and the coarse matrix G^T G.
//
// Bilinear forms of Sec. 2.3, Eqs. (2.21)-(2.23), with the 3-field elimination of eta
// (W_h = M_h^P, Sec. 2.4, so the eta row of Eq. (2.43) gives eta = (p - k1 xi)/k2 exactly):
//   (u,u)   a(u,v)   = 2 mu (eps u, eps v) = mu sum_q [d_cd grad phi_i . grad phi_j + d_d phi_i d_c phi_j]
//   (xi,u)  b(v,xi)  = -(xi, div v)
//   (xi,xi) -R/lambda,  (xi,p) (alpha/lambda) R,  (p,p) -((c0 + alpha^2/lambda) R + tau A_f)
// On affine triangles every integrand is a polynomial of degree <= 2, integrated exactly by
// the edge-midpoint rule.  Loads use the symmetric 7-point rule of degree 5 (Radon 1948).
// The mesh is structured, so a subdomain has two triangle shapes: their element matrices
// are computed once per subdomain in shared memory.  Scatter is race-free and deterministic:
// cells are processed in 4 colours (i % 2, j % 2) with a block barrier between colours.
#include <cmath>

#include "device.cuh"

namespace fp {

namespace {

__device__ __forceinline__ double sq(double v) { return v * v; }

// ---- closed-form data of Test Case 1 (Sec. 4.1), own restatement ---------------------
struct Mf {
  double lam, mu, alpha, c0, K, mu_f;
  __device__ double beta() const { return alpha / (lam + 2.0 * mu); }
  __device__ void f_P(double x, double y, double &fx, double &fy) const {
    const double PI = 3.141592653589793238462643383279502884;
    const double s = sin(2 * PI * x) * sin(2 * PI * y), c = cos(2 * PI * x) * cos(2 * PI * y);
    const double v = 8 * PI * PI * mu * s - 4 * PI * PI * (lam + mu) * (c - s);
    fx = v + alpha * PI * cos(PI * x) * sin(PI * y);
    fy = v + alpha * PI * sin(PI * x) * cos(PI * y);
  }
  __device__ void f_E(double x, double y, double &fx, double &fy) const {
    const double PI = 3.141592653589793238462643383279502884;
    const double s = sin(2 * PI * x) * sin(2 * PI * y), c = cos(2 * PI * x) * cos(2 * PI * y);
    const double v = 8 * PI * PI * mu * s - 4 * PI * PI * (lam + mu) * (c - s);
    const double q = sin(PI * x) * sin(PI * y);
    const double qx = PI * cos(PI * x) * sin(PI * y);
    const double qy = PI * sin(PI * x) * cos(PI * y);
    const double qxy = PI * PI * cos(PI * x) * cos(PI * y);
    const double bt = beta(), ym = y - 0.5;
    const double g_xy = -bt * (qxy * ym + qx);
    const double g_yy = bt * PI * PI * q * ym - 2 * bt * qy;
    const double lap_g = 2 * bt * PI * PI * q * ym - 2 * bt * qy;
    fx = v - (lam + mu) * g_xy;
    fy = v - mu * lap_g - (lam + mu) * g_yy;
  }
  __device__ double z(double x, double y) const {
    const double PI = 3.141592653589793238462643383279502884;
    return (K / mu_f) * 2 * PI * PI * sin(PI * x) * sin(PI * y);
  }
  __device__ double eta0(double x, double y) const {
    // eta_0 = c0 p_0 + alpha div u_0
    const double PI = 3.141592653589793238462643383279502884;
    const double div = 2 * PI * (cos(2 * PI * x) * sin(2 * PI * y) + sin(2 * PI * x) * cos(2 * PI * y));
    return c0 * sin(PI * x) * sin(PI * y) + alpha * div;
  }
};

// element shape data of triangle type tt on a cell of size hx x hy
__device__ void tri_vertices(int tt, double hx, double hy, double v[3][2]) {
  v[0][0] = 0; v[0][1] = 0;
  if (tt == 0) { v[1][0] = hx; v[1][1] = 0; v[2][0] = hx; v[2][1] = hy; }
  else { v[1][0] = hx; v[1][1] = hy; v[2][0] = 0; v[2][1] = hy; }
}

__device__ void bary_grad(const double v[3][2], double G[3][2], double &area) {
  const double bx = v[1][0] - v[0][0], by = v[1][1] - v[0][1];
  const double cx = v[2][0] - v[0][0], cy = v[2][1] - v[0][1];
  const double det = bx * cy - by * cx;
  G[1][0] = cy / det; G[1][1] = -cx / det;
  G[2][0] = -by / det; G[2][1] = bx / det;
  G[0][0] = -G[1][0] - G[2][0]; G[0][1] = -G[1][1] - G[2][1];
  area = 0.5 * fabs(det);
}

// gradient of displacement basis function i (P_k) at barycentric point L
__device__ void grad_phi(int k, int i, const double L[3], const double G[3][2], double g[2]) {
  if (k == 1) { g[0] = G[i][0]; g[1] = G[i][1]; return; }
  if (i < 3) {
    const double s = 4 * L[i] - 1;
    g[0] = s * G[i][0]; g[1] = s * G[i][1];
    return;
  }
  const int a = (i == 3) ? 0 : (i == 4 ? 1 : 2);
  const int b = (i == 3) ? 1 : (i == 4 ? 2 : 0);
  g[0] = 4 * (L[a] * G[b][0] + L[b] * G[a][0]);
  g[1] = 4 * (L[a] * G[b][1] + L[b] * G[a][1]);
}

__device__ double phi(int k, int i, const double L[3]) {
  if (k == 1 || i < 3) return k == 1 ? L[i] : L[i] * (2 * L[i] - 1);
  const int a = (i == 3) ? 0 : (i == 4 ? 1 : 2);
  const int b = (i == 3) ? 1 : (i == 4 ? 2 : 0);
  return 4 * L[a] * L[b];
}

__device__ int csr_find(const int *col, int lo, int hi, int c) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (col[mid] < c) lo = mid + 1; else hi = mid;
  }
  return lo;
}

}  // namespace

// One CTA per subdomain.  Shared memory: element matrices of both triangle types.
__global__ void k_assemble(DevTopo T, DevParams P, double *csr_val, double *fstat, double *Zn,
                           double *E0n) {
  const int s = blockIdx.x;
  const DevTpl t = T.tpl[T.sub_tpl[s]];
  const int k = t.k, nun = k == 1 ? 3 : 6, nu = 2 * nun;
  __shared__ double Ae[2][12][12], Be[2][3][12], Re[2][3][3], Afe[2][3][3];
  const double hx = T.sub_hx[s], hy = T.sub_hy[s];
  const double x0 = T.sub_x0[s], y0 = T.sub_y0[s];
  // --- phase 1: element matrices of the two triangle shapes --------------------------
  const double Lq[3][3] = {{0.5, 0.5, 0.0}, {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}};
  for (int e = threadIdx.x; e < 2 * (nu * nu + 3 * nu + 18); e += blockDim.x) {
    const int per = nu * nu + 3 * nu + 18;
    const int tt = e / per;
    int r = e % per;
    double v[3][2], G[3][2], area;
    tri_vertices(tt, hx, hy, v);
    bary_grad(v, G, area);
    if (r < nu * nu) {
      const int a = r / nu, b = r % nu;
      const int i = a / 2, c = a % 2, j = b / 2, d = b % 2;
      double acc = 0;
      for (int q = 0; q < 3; ++q) {
        double gi[2], gj[2];
        grad_phi(k, i, Lq[q], G, gi);
        grad_phi(k, j, Lq[q], G, gj);
        acc += (c == d ? gi[0] * gj[0] + gi[1] * gj[1] : 0.0) + gi[d] * gj[c];
      }
      Ae[tt][a][b] = P.mu * area / 3.0 * acc;
      continue;
    }
    r -= nu * nu;
    if (r < 3 * nu) {
      const int m = r / nu, b = r % nu, j = b / 2, d = b % 2;
      double acc = 0;
      for (int q = 0; q < 3; ++q) {
        double gj[2];
        grad_phi(k, j, Lq[q], G, gj);
        acc += Lq[q][m] * gj[d];
      }
      Be[tt][m][b] = -area / 3.0 * acc;
      continue;
    }
    r -= 3 * nu;
    if (r < 9) {
      const int m = r / 3, n2 = r % 3;
      Re[tt][m][n2] = area * (m == n2 ? 2.0 : 1.0) / 12.0;
    } else {
      r -= 9;
      const int m = r / 3, n2 = r % 3;
      Afe[tt][m][n2] = area * (G[m][0] * G[n2][0] + G[m][1] * G[n2][1]) / P.mu_f;
    }
  }
  __syncthreads();
  // --- phase 2: scatter, 4 colours ---------------------------------------------------
  const int *ed_all = T.pool + t.elem_dofs;
  const int *cptr = T.pool + t.csr_ptr, *ccol = T.pool + t.csr_col;
  double *val = csr_val + T.csr_off[s];
  double *fs = fstat + T.vec_off[s];
  const long long pn0 = T.pnode_off[s];
  const double lam = P.lam, al = P.alpha;
  const double cxi = -1.0 / lam, cxp = al / lam, cpp = -(P.c0 + al * al / lam);
  const Mf mf{P.lam, P.mu, P.alpha, P.c0, P.perm_k, P.mu_f};
  // 7-point degree-5 rule
  const double s15 = sqrt(15.0);
  const double a1 = (6.0 - s15) / 21.0, a2 = (6.0 + s15) / 21.0;
  const double w0 = 9.0 / 40.0, w1 = (155.0 - s15) / 1200.0, w2 = (155.0 + s15) / 1200.0;
  const double QL[7][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3},
                           {1 - 2 * a1, a1, a1}, {a1, 1 - 2 * a1, a1}, {a1, a1, 1 - 2 * a1},
                           {1 - 2 * a2, a2, a2}, {a2, 1 - 2 * a2, a2}, {a2, a2, 1 - 2 * a2}};
  const double QW[7] = {w0, w1, w1, w1, w2, w2, w2};
  const int nx = t.nx, ny = t.ny;
  for (int color = 0; color < 4; ++color) {
    const int ci = color & 1, cj = color >> 1;
    const int ncx = (nx - ci + 1) / 2, ncy = (ny - cj + 1) / 2;
    for (int cell = threadIdx.x; cell < ncx * ncy; cell += blockDim.x) {
      const int i = ci + 2 * (cell % ncx), j = cj + 2 * (cell / ncx);
      for (int tt = 0; tt < 2; ++tt) {
        const int e = 2 * (j * nx + i) + tt;
        const int *ed = ed_all + (long long)e * t.ndl;
        const double Ke = P.perm ? P.perm[T.elem_off[s] + e] : P.perm_k;
        // matrix entries
        for (int a = 0; a < t.ndl; ++a) {
          const int ra = ed[a];
          if (ra < 0) continue;
          const int lo = cptr[ra], hi = cptr[ra + 1];
          for (int b = 0; b < t.ndl; ++b) {
            const int cb = ed[b];
            if (cb < 0) continue;
            double v;
            if (a < nu && b < nu) v = Ae[tt][a][b];
            else if (a < nu) { if (b < nu + 3) v = Be[tt][b - nu][a]; else continue; }
            else if (b < nu) { if (a < nu + 3) v = Be[tt][a - nu][b]; else continue; }
            else {
              const int ma = a - nu, mb = b - nu;
              if (ma < 3 && mb < 3) v = cxi * Re[tt][ma][mb];
              else if (ma < 3) v = cxp * Re[tt][ma][mb - 3];
              else if (mb < 3) v = cxp * Re[tt][ma - 3][mb];
              else v = cpp * Re[tt][ma - 3][mb - 3] - P.tau * Ke * Afe[tt][ma - 3][mb - 3];
            }
            const int pos = csr_find(ccol, lo, hi, cb);
            val[pos] += v;
          }
        }
        // loads (manufactured solution; the point source enters per step)
        if (P.source != 1) {
          double vv[3][2], G[3][2], area;
          tri_vertices(tt, hx, hy, vv);
          bary_grad(vv, G, area);
          const double ox = x0 + i * hx, oy = y0 + j * hy;
          double Fl[12] = {0}, Zl[3] = {0}, El[3] = {0};
          for (int q = 0; q < 7; ++q) {
            const double X = ox + QL[q][0] * vv[0][0] + QL[q][1] * vv[1][0] + QL[q][2] * vv[2][0];
            const double Y = oy + QL[q][0] * vv[0][1] + QL[q][1] * vv[1][1] + QL[q][2] * vv[2][1];
            double fx, fy;
            if (t.poro) mf.f_P(X, Y, fx, fy); else mf.f_E(X, Y, fx, fy);
            const double wa = QW[q] * area;
            for (int nI = 0; nI < nun; ++nI) {
              const double ph = phi(k, nI, QL[q]);
              Fl[2 * nI] += wa * fx * ph;
              Fl[2 * nI + 1] += wa * fy * ph;
            }
            if (t.poro) {
              const double zz = mf.z(X, Y), e0 = mf.eta0(X, Y);
              for (int m = 0; m < 3; ++m) { Zl[m] += wa * zz * QL[q][m]; El[m] += wa * e0 * QL[q][m]; }
            }
          }
          for (int a = 0; a < nu; ++a)
            if (ed[a] >= 0) fs[ed[a]] += Fl[a];
          if (t.poro) {
            const int v00 = j * t.npx + i;
            const int vi0 = v00, vi1 = tt == 0 ? v00 + 1 : v00 + t.npx + 1, vi2 = tt == 0 ? v00 + t.npx + 1 : v00 + t.npx;
            Zn[pn0 + vi0] += Zl[0]; Zn[pn0 + vi1] += Zl[1]; Zn[pn0 + vi2] += Zl[2];
            E0n[pn0 + vi0] += El[0]; E0n[pn0 + vi1] += El[1]; E0n[pn0 + vi2] += El[2];
          }
        }
      }
    }
    __syncthreads();
  }
}

// R eta^0 from given initial fields (Sec. 2.5, eta_0 = c0 p_0 + alpha div u_0 by Eq. 2.17):
// Reta[v] = sum over elements of int (c0 p0_h + alpha div u0_h) phi_v, with u0_h the P_k
// interpolant of the nodal u0 (every node, Dirichlet ones included) and p0_h the P1
// interpolant of p0; the integrand has degree <= 2, so the edge-midpoint rule is exact.
// u0, p0: canonical node arrays (may be null: zero).  One CTA per poroelastic subdomain,
// cells in 4 colours as in the assembly (race-free, fixed order).
__global__ void k_set_initial(DevTopo T, DevParams P, const double *u0, const double *p0, double *Reta) {
  const int s = blockIdx.x;
  const DevTpl t = T.tpl[T.sub_tpl[s]];
  const long long pn0 = T.pnode_off[s], un0 = T.unode_off[s];
  for (int v = threadIdx.x; v < t.npx * t.npy; v += blockDim.x) Reta[pn0 + v] = 0.0;
  __syncthreads();
  if (!t.poro) return;
  const int k = t.k, nun = k == 1 ? 3 : 6, nx = t.nx, ny = t.ny;
  const double hx = T.sub_hx[s], hy = T.sub_hy[s];
  const double Lq[3][3] = {{0.5, 0.5, 0.0}, {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}};
  for (int color = 0; color < 4; ++color) {
    const int ci = color & 1, cj = color >> 1;
    const int ncx = (nx - ci + 1) / 2, ncy = (ny - cj + 1) / 2;
    for (int cell = threadIdx.x; cell < ncx * ncy; cell += blockDim.x) {
      const int i = ci + 2 * (cell % ncx), j = cj + 2 * (cell / ncx);
      for (int tt = 0; tt < 2; ++tt) {
        double vv[3][2], G[3][2], area;
        tri_vertices(tt, hx, hy, vv);
        bary_grad(vv, G, area);
        // vertex offsets in cell units: type 0 (0,0),(1,0),(1,1); type 1 (0,0),(1,1),(0,1)
        const int ox[3] = {0, 1, tt == 0 ? 1 : 0}, oy[3] = {0, tt == 0 ? 0 : 1, 1};
        // P1 vertices (pressure grid) and P_k nodes (displacement grid, x fastest)
        int pv[3], un[6];
        for (int a = 0; a < 3; ++a) {
          pv[a] = (j + oy[a]) * t.npx + (i + ox[a]);
          un[a] = (k * (j + oy[a])) * t.nux + k * (i + ox[a]);
        }
        if (k == 2) {
          const int ea[3] = {0, 1, 2}, eb[3] = {1, 2, 0};
          for (int m = 0; m < 3; ++m) {
            const int gx = (2 * (i + ox[ea[m]]) + 2 * (i + ox[eb[m]])) / 2;
            const int gy = (2 * (j + oy[ea[m]]) + 2 * (j + oy[eb[m]])) / 2;
            un[3 + m] = gy * t.nux + gx;
          }
        }
        double El[3] = {0.0, 0.0, 0.0};
        for (int q = 0; q < 3; ++q) {
          double pq = 0.0, div = 0.0;
          if (p0)
            for (int a = 0; a < 3; ++a) pq += Lq[q][a] * p0[pn0 + pv[a]];
          if (u0)
            for (int a = 0; a < nun; ++a) {
              double g[2];
              grad_phi(k, a, Lq[q], G, g);
              div += g[0] * u0[2 * (un0 + un[a])] + g[1] * u0[2 * (un0 + un[a]) + 1];
            }
          const double eta = P.c0 * pq + P.alpha * div;
          for (int m = 0; m < 3; ++m) El[m] += area / 3.0 * eta * Lq[q][m];
        }
        for (int m = 0; m < 3; ++m) Reta[pn0 + pv[m]] += El[m];
      }
    }
    __syncthreads();
  }
}

// Band matrix (cyclic column layout, see band.cu) from the CSR values.  mode 0: Neumann
// (identity rows on the fixed dofs of floating subdomains); mode 1: Dirichlet (identity rows
// on every dof touched by B_s).  One CTA per subdomain.
template <typename T>
__global__ void k_csr_to_band(DevTopo D, const double *csr_val, T *band, int mode) {
  const int s = blockIdx.x;
  const DevTpl t = D.tpl[D.sub_tpl[s]];
  T *A = band + D.fac_off[s];
  const long long tot = (long long)t.n * t.LD;
  for (long long e = threadIdx.x; e < tot; e += blockDim.x) A[e] = T(0);
  __syncthreads();
  const int *cptr = D.pool + t.csr_ptr, *ccol = D.pool + t.csr_col;
  const int *isb = D.pool + t.is_bnd;
  const double *val = csr_val + D.csr_off[s];
  auto ident = [&](int d) {
    if (mode == 1) return isb[d] != 0;
    return t.floating && (d == t.fixed0 || d == t.fixed1 || d == t.fixed2);
  };
  for (int r = threadIdx.x; r < t.n; r += blockDim.x) {
    const bool ir = ident(r);
    if (ir) { A[(long long)r * t.LD + r % t.LD] = T(1); continue; }
    for (int e = cptr[r]; e < cptr[r + 1]; ++e) {
      const int c = ccol[e];
      if (c > r || ident(c)) continue;
      A[(long long)c * t.LD + r % t.LD] = T(val[e]);
    }
  }
}

cudaError_t launch_csr_to_band(bool fp32, DevTopo D, const double *csr_val, void *band, int mode, cudaStream_t s) {
  if (fp32) k_csr_to_band<float><<<D.S, 256, 0, s>>>(D, csr_val, (float *)band, mode);
  else k_csr_to_band<double><<<D.S, 256, 0, s>>>(D, csr_val, (double *)band, mode);
  return cudaGetLastError();
}

// Rows of G = [B_s R_s] (FETI-1 coarse space; rigid modes (1,0), (0,1), (-(y-yc), x-xc)/L).
__global__ void k_coarse_G(DevTopo D, double *ga, double *gb) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= D.nlam) return;
  for (int side = 0; side < 2; ++side) {
    const int s = side == 0 ? D.lam_sa[r] : D.lam_sb[r];
    const int d = side == 0 ? D.lam_da[r] : D.lam_db[r];
    double *g = (side == 0 ? ga : gb) + 3 * (long long)r;
    g[0] = g[1] = g[2] = 0.0;
    if (D.sub_float[s] < 0) continue;
    const DevTpl t = D.tpl[D.sub_tpl[s]];
    const int field = D.pool[t.dof_field + d];
    if (field > 1) continue;
    const int node = D.pool[t.dof_node + d];
    const double hx = D.sub_hx[s], hy = D.sub_hy[s];
    // the same arithmetic as the rigid modes of the right-hand side and the recovery
    const double hxk = hx / t.k, hyk = hy / t.k, invL = 1.0 / fmax(t.nx * hx, t.ny * hy);
    const double x = D.sub_x0[s] + (node % t.nux) * hxk;
    const double y = D.sub_y0[s] + (node / t.nux) * hyk;
    const double xc = D.sub_x0[s] + 0.5 * t.nx * hx, yc = D.sub_y0[s] + 0.5 * t.ny * hy;
    const double sg = side == 0 ? 1.0 : -1.0;
    if (field == 0) { g[0] = sg; g[2] = -sg * (y - yc) * invL; }
    else { g[1] = sg; g[2] = sg * (x - xc) * invL; }
  }
}

// G^T G in the band layout of band.cu; one thread per floating subdomain owns its block row.
__global__ void k_coarse_GtG(DevTopo D, const double *ga, const double *gb, double *H) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= D.NF) return;
  constexpr int MAXNB = 16;
  int nb_id[MAXNB];
  double blk[MAXNB][9];
  int nnb = 0;
  double diag[9] = {0};
  for (int q = D.float_rows_ptr[f]; q < D.float_rows_ptr[f + 1]; ++q) {
    const int r = D.float_rows[q];
    const bool mine_a = D.lam_fa[r] == f;
    const double *gf = (mine_a ? ga : gb) + 3 * (long long)r;
    const double *go = (mine_a ? gb : ga) + 3 * (long long)r;
    const int o = mine_a ? D.lam_fb[r] : D.lam_fa[r];
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) diag[3 * a + c] += gf[a] * gf[c];
    if (o >= 0 && o < f) {
      int slot = -1;
      for (int z = 0; z < nnb; ++z) if (nb_id[z] == o) slot = z;
      if (slot < 0 && nnb < MAXNB) {
        slot = nnb++;
        nb_id[slot] = o;
        for (int z = 0; z < 9; ++z) blk[slot][z] = 0.0;
      }
      if (slot >= 0)
        for (int a = 0; a < 3; ++a)
          for (int c = 0; c < 3; ++c) blk[slot][3 * a + c] += gf[a] * go[c];
    }
  }
  const int LD = D.LDH;
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c <= a; ++c) {
      const int row = 3 * f + a, col = 3 * f + c;
      H[(long long)col * LD + row % LD] = diag[3 * a + c];
    }
  for (int z = 0; z < nnb; ++z)
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) {
        const int row = 3 * f + a, col = 3 * nb_id[z] + c;
        H[(long long)col * LD + row % LD] = blk[z][3 * a + c];
      }
}

}  // namespace fp
