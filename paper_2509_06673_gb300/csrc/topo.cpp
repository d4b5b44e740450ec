// Host-side topology: dof numbering in band order, sparsity patterns, interface tables.
//
// Sec. 2.4 (finite element spaces) and Sec. 3.1 (the reordered local systems) define
// what is numbered; the band ordering itself is this library's choice: displacement nodes
// are visited row by row along the shorter side of the subdomain, and at every node its
// displacement dofs, then (at P1 vertices) xi and p.  The local 3-field matrices are
// symmetric quasi-definite, so LDL^T needs no pivoting in any ordering.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cstring>
#include <exception>
#include <map>
#include <thread>
#include <tuple>

#include "internal.h"

namespace fp {

namespace {

int round_up(int v, int m) { return (v + m - 1) / m * m; }

void build_template(Template &t) {
  const int k = t.k;
  t.nux = k * t.nx + 1;
  t.nuy = k * t.ny + 1;
  t.npx = t.nx + 1;
  t.npy = t.ny + 1;
  t.transposed = t.nx > t.ny ? 1 : 0;
  t.floating = 1;
  for (int q = 0; q < 4; ++q)
    if (t.side_u[q] == SU_CLAMPED) t.floating = 0;
  const int NU = t.nux * t.nuy, NP = t.npx * t.npy;
  auto u_dir = [&](int I, int J) {
    return (I == 0 && t.side_u[0] == SU_CLAMPED) || (I == t.nux - 1 && t.side_u[1] == SU_CLAMPED) ||
           (J == 0 && t.side_u[2] == SU_CLAMPED) || (J == t.nuy - 1 && t.side_u[3] == SU_CLAMPED);
  };
  auto u_bnd = [&](int I, int J) {
    if (u_dir(I, J)) return false;
    return (I == 0 && t.side_u[0] == SU_IFACE) || (I == t.nux - 1 && t.side_u[1] == SU_IFACE) ||
           (J == 0 && t.side_u[2] == SU_IFACE) || (J == t.nuy - 1 && t.side_u[3] == SU_IFACE);
  };
  auto p_dir = [&](int i, int j) {
    if (!t.poro) return true;
    return (i == 0 && t.side_p[0] == SP_DIRICHLET) || (i == t.npx - 1 && t.side_p[1] == SP_DIRICHLET) ||
           (j == 0 && t.side_p[2] == SP_DIRICHLET) || (j == t.npy - 1 && t.side_p[3] == SP_DIRICHLET);
  };
  auto p_bnd = [&](int i, int j) {
    if (p_dir(i, j)) return false;
    return (i == 0 && t.side_p[0] == SP_IFACE) || (i == t.npx - 1 && t.side_p[1] == SP_IFACE) ||
           (j == 0 && t.side_p[2] == SP_IFACE) || (j == t.npy - 1 && t.side_p[3] == SP_IFACE);
  };
  t.udof.assign(2 * NU, -1);
  t.xidof.assign(NP, -1);
  t.pdof.assign(NP, -1);
  t.dof_field.clear();
  t.dof_node.clear();
  std::vector<uint8_t> bnd_flag;
  int n = 0;
  const int outer = t.transposed ? t.nux : t.nuy;
  const int inner = t.transposed ? t.nuy : t.nux;
  for (int o = 0; o < outer; ++o) {
    for (int in = 0; in < inner; ++in) {
      const int I = t.transposed ? o : in;
      const int J = t.transposed ? in : o;
      const int a = J * t.nux + I;
      if (!u_dir(I, J)) {
        const bool bd = u_bnd(I, J);
        for (int c = 0; c < 2; ++c) {
          t.udof[2 * a + c] = n++;
          t.dof_field.push_back(c);
          t.dof_node.push_back(a);
          bnd_flag.push_back(bd);
        }
      }
      if (I % k == 0 && J % k == 0) {
        const int i = I / k, j = J / k, b = j * t.npx + i;
        t.xidof[b] = n++;
        t.dof_field.push_back(F_XI);
        t.dof_node.push_back(b);
        bnd_flag.push_back(0);
        if (t.poro && !p_dir(i, j)) {
          t.pdof[b] = n++;
          t.dof_field.push_back(F_P);
          t.dof_node.push_back(b);
          bnd_flag.push_back(p_bnd(i, j));
        }
      }
    }
  }
  t.n = n;
  t.is_bnd = bnd_flag;
  t.bnd.clear();
  for (int d = 0; d < n; ++d)
    if (bnd_flag[d]) t.bnd.push_back(d);
  // elements: cell (i, j), triangles t=0 (v00, v10, v11), t=1 (v00, v11, v01)
  const int nun = k == 1 ? 3 : 6;
  t.ndl = 2 * nun + 3 + (t.poro ? 3 : 0);
  const int ne = 2 * t.nx * t.ny;
  t.elem_dofs.assign((size_t)ne * t.ndl, -1);
  int bmax = 0;
  for (int j = 0; j < t.ny; ++j) {
    for (int i = 0; i < t.nx; ++i) {
      for (int tt = 0; tt < 2; ++tt) {
        int un[6], vi[3];
        const int v00 = j * t.npx + i, v10 = v00 + 1, v01 = v00 + t.npx, v11 = v01 + 1;
        if (tt == 0) { vi[0] = v00; vi[1] = v10; vi[2] = v11; }
        else { vi[0] = v00; vi[1] = v11; vi[2] = v01; }
        auto U = [&](int I, int J) { return J * t.nux + I; };
        if (k == 1) {
          if (tt == 0) { un[0] = U(i, j); un[1] = U(i + 1, j); un[2] = U(i + 1, j + 1); }
          else { un[0] = U(i, j); un[1] = U(i + 1, j + 1); un[2] = U(i, j + 1); }
        } else {
          const int I = 2 * i, J = 2 * j;
          if (tt == 0) {
            un[0] = U(I, J); un[1] = U(I + 2, J); un[2] = U(I + 2, J + 2);
            un[3] = U(I + 1, J); un[4] = U(I + 2, J + 1); un[5] = U(I + 1, J + 1);
          } else {
            un[0] = U(I, J); un[1] = U(I + 2, J + 2); un[2] = U(I, J + 2);
            un[3] = U(I + 1, J + 1); un[4] = U(I + 1, J + 2); un[5] = U(I, J + 1);
          }
        }
        int *ed = &t.elem_dofs[(size_t)(2 * (j * t.nx + i) + tt) * t.ndl];
        for (int q = 0; q < nun; ++q) {
          ed[2 * q] = t.udof[2 * un[q]];
          ed[2 * q + 1] = t.udof[2 * un[q] + 1];
        }
        for (int q = 0; q < 3; ++q) ed[2 * nun + q] = t.xidof[vi[q]];
        if (t.poro)
          for (int q = 0; q < 3; ++q) ed[2 * nun + 3 + q] = t.pdof[vi[q]];
        int lo = 1 << 30, hi = -1;
        for (int q = 0; q < t.ndl; ++q)
          if (ed[q] >= 0) { lo = std::min(lo, ed[q]); hi = std::max(hi, ed[q]); }
        if (hi >= 0) bmax = std::max(bmax, hi - lo);
      }
    }
  }
  t.b = bmax;
  t.LD = round_up(bmax + 1, 32);
  // CSR pattern: every (row, column) pair of every element, counted, filled, then sorted
  // and made unique per row
  std::vector<int> cnt(n + 1, 0);
  for (int e = 0; e < ne; ++e) {
    const int *ed = &t.elem_dofs[(size_t)e * t.ndl];
    int valid = 0;
    for (int c = 0; c < t.ndl; ++c) valid += ed[c] >= 0;
    for (int a = 0; a < t.ndl; ++a)
      if (ed[a] >= 0) cnt[ed[a] + 1] += valid;
  }
  for (int r = 0; r < n; ++r) cnt[r + 1] += cnt[r];
  std::vector<int> all(cnt[n]), fill(cnt.begin(), cnt.end() - 1);
  for (int e = 0; e < ne; ++e) {
    const int *ed = &t.elem_dofs[(size_t)e * t.ndl];
    for (int a = 0; a < t.ndl; ++a) {
      if (ed[a] < 0) continue;
      for (int c = 0; c < t.ndl; ++c)
        if (ed[c] >= 0) all[fill[ed[a]]++] = ed[c];
    }
  }
  t.csr_ptr.assign(n + 1, 0);
  t.csr_col.clear();
  t.csr_col.reserve(cnt[n]);
  for (int r = 0; r < n; ++r) {
    int *b0 = all.data() + cnt[r], *b1 = all.data() + cnt[r + 1];
    std::sort(b0, b1);
    b1 = std::unique(b0, b1);
    t.csr_ptr[r + 1] = t.csr_ptr[r] + (int)(b1 - b0);
    t.csr_col.insert(t.csr_col.end(), b0, b1);
  }
  // halo rows for the Dirichlet preconditioner
  t.halo_ptr.assign(1, 0);
  t.halo_row.clear();
  t.halo_ent.clear();
  for (int r = 0; r < n; ++r) {
    if (t.is_bnd[r]) continue;
    int cnt = 0;
    for (int e = t.csr_ptr[r]; e < t.csr_ptr[r + 1]; ++e)
      if (t.is_bnd[t.csr_col[e]]) { t.halo_ent.push_back(e); ++cnt; }
    if (cnt) {
      t.halo_row.push_back(r);
      t.halo_ptr.push_back((int)t.halo_ent.size());
    }
  }
  // fixed dofs for the generalised inverse of a floating subdomain
  t.fixed[0] = t.fixed[1] = t.fixed[2] = -1;
  if (t.floating) {
    t.fixed[0] = t.udof[0];
    t.fixed[1] = t.udof[1];
    t.fixed[2] = t.udof[2 * (t.nux - 1) + 1];
  }
  // sliced ELL (32-row slices, column-major inside a slice) of the Neumann matrix
  auto is_fixed = [&](int d) { return t.floating && (d == t.fixed[0] || d == t.fixed[1] || d == t.fixed[2]); };
  const int nslice = (n + 31) / 32;
  t.sell_ptr.assign(nslice + 1, 0);
  t.sell_col.clear();
  t.sell_src.clear();
  for (int q = 0; q < nslice; ++q) {
    // entries of row 32 q + l: (col, CSR index) of its non-fixed columns, or (r, -2) on a
    // fixed row; slot k of the row at base + 32 k + l, padding (min(r, n - 1), -1)
    int len[32], w = 0;
    for (int l = 0; l < 32; ++l) {
      const int r = 32 * q + l;
      len[l] = 0;
      if (r >= n) continue;
      if (is_fixed(r)) {
        len[l] = 1;
      } else {
        for (int e = t.csr_ptr[r]; e < t.csr_ptr[r + 1]; ++e) len[l] += !is_fixed(t.csr_col[e]);
      }
      w = std::max(w, len[l]);
    }
    const size_t base = t.sell_col.size();
    t.sell_col.resize(base + (size_t)32 * w);
    t.sell_src.resize(base + (size_t)32 * w);
    for (int l = 0; l < 32; ++l) {
      const int r = 32 * q + l;
      int k2 = 0;
      if (r < n) {
        if (is_fixed(r)) {
          t.sell_col[base + l] = r;
          t.sell_src[base + l] = -2;
          k2 = 1;
        } else {
          for (int e = t.csr_ptr[r]; e < t.csr_ptr[r + 1]; ++e) {
            if (is_fixed(t.csr_col[e])) continue;
            t.sell_col[base + (size_t)32 * k2 + l] = t.csr_col[e];
            t.sell_src[base + (size_t)32 * k2 + l] = e;
            ++k2;
          }
        }
      }
      for (; k2 < w; ++k2) {
        t.sell_col[base + (size_t)32 * k2 + l] = std::min(r, n - 1);
        t.sell_src[base + (size_t)32 * k2 + l] = -1;
      }
    }
    t.sell_ptr[q + 1] = (int)t.sell_col.size();
  }
}

// Builds every template; templates are independent, so they are built by a small pool of
// host threads pulling indices from a shared counter (an uneven partition has one template
// per distinct subdomain shape, about a thousand for a 32 x 32 partition).  The result does
// not depend on the number of threads.  An exception in a worker is rethrown here.
void build_templates(std::vector<Template> &tpl) {
  const int nt = (int)tpl.size();
  const int hw = (int)std::thread::hardware_concurrency();
  const int nth = std::max(1, std::min(std::min(nt, 32), hw > 0 ? hw : 1));
  std::atomic<int> next(0);
  std::vector<std::exception_ptr> errs(nth);
  auto work = [&](int w) {
    try {
      for (int i = next.fetch_add(1); i < nt; i = next.fetch_add(1)) build_template(tpl[i]);
    } catch (...) {
      errs[w] = std::current_exception();
      next.store(nt);
    }
  };
  std::vector<std::thread> pool;
  for (int w = 1; w < nth; ++w) {
    try {
      pool.emplace_back(work, w);
    } catch (...) {
      break;  // fewer threads: the remaining indices are taken by the others
    }
  }
  work(0);
  for (auto &th : pool) th.join();
  for (auto &e : errs)
    if (e) std::rethrow_exception(e);
}

struct NodeEnt { int s, d0, d1; };

}  // namespace

bool build_topology(const fp_mesh_desc *m, const fp_params *p, Topology &T, std::string &err) {
  if (!m || !p) { err = "null mesh or params"; return false; }
  if (m->nsub_x < 1 || m->nsub_y < 2 || !m->cells_x || !m->cells_y) { err = "bad partition"; return false; }
  // global node indices (k * sum of cells + 1 per direction) and the subdomain count stay in int
  if (m->nsub_x > 4096 || m->nsub_y > 4096) { err = "nsub_x and nsub_y must be at most 4096"; return false; }
  if (m->order_k != 1 && m->order_k != 2) { err = "order_k must be 1 or 2"; return false; }
  if (m->poro_rows < 1 || m->poro_rows >= m->nsub_y) { err = "poro_rows must be in [1, nsub_y)"; return false; }
  T.nsx = m->nsub_x; T.nsy = m->nsub_y; T.poro_rows = m->poro_rows; T.k = m->order_k;
  T.S = T.nsx * T.nsy;
  T.cells_x.assign(m->cells_x, m->cells_x + T.nsx);
  T.cells_y.assign(m->cells_y, m->cells_y + T.nsy);
  for (int c : T.cells_x) if (c < 1 || c > 4096) { err = "cells_x out of range"; return false; }
  for (int c : T.cells_y) if (c < 1 || c > 4096) { err = "cells_y out of range"; return false; }
  const int S = T.S, k = T.k;
  std::map<std::vector<int>, int> tpl_index;
  T.tpl.clear();
  T.sub_tpl.assign(S, -1);
  T.sub_x0.resize(S); T.sub_y0.resize(S); T.sub_hx.resize(S); T.sub_hy.resize(S);
  T.sub_I0.resize(S); T.sub_J0.resize(S); T.sub_i0.resize(S); T.sub_j0.resize(S);
  std::vector<int> cxs(T.nsx + 1, 0), cys(T.nsy + 1, 0);
  for (int c = 0; c < T.nsx; ++c) cxs[c + 1] = cxs[c] + T.cells_x[c];
  for (int c = 0; c < T.nsy; ++c) cys[c + 1] = cys[c] + T.cells_y[c];
  for (int s = 0; s < S; ++s) {
    const int cx = s % T.nsx, cy = s / T.nsx;
    const int poro = cy < T.poro_rows;
    int su[4] = {cx == 0 ? SU_CLAMPED : SU_IFACE, cx == T.nsx - 1 ? SU_CLAMPED : SU_IFACE,
                 cy == 0 ? SU_CLAMPED : SU_IFACE, cy == T.nsy - 1 ? SU_CLAMPED : SU_IFACE};
    int sp[4] = {SP_NATURAL, SP_NATURAL, SP_NATURAL, SP_NATURAL};
    if (poro) {
      sp[0] = cx == 0 ? SP_DIRICHLET : SP_IFACE;
      sp[1] = cx == T.nsx - 1 ? SP_DIRICHLET : SP_IFACE;
      sp[2] = cy == 0 ? SP_DIRICHLET : SP_IFACE;
      sp[3] = cy == T.poro_rows - 1 ? SP_NATURAL : SP_IFACE;
    }
    const int nx = T.cells_x[cx], ny = T.cells_y[cy];
    std::vector<int> key = {nx, ny, k, poro, su[0], su[1], su[2], su[3], sp[0], sp[1], sp[2], sp[3]};
    auto it = tpl_index.find(key);
    int ti;
    if (it == tpl_index.end()) {
      Template t;  // numbered in first-use order; built below
      t.nx = nx; t.ny = ny; t.k = k; t.poro = poro;
      std::memcpy(t.side_u, su, sizeof su);
      std::memcpy(t.side_p, sp, sizeof sp);
      ti = (int)T.tpl.size();
      T.tpl.push_back(std::move(t));
      tpl_index[key] = ti;
    } else {
      ti = it->second;
    }
    T.sub_tpl[s] = ti;
    T.sub_x0[s] = (double)cx / T.nsx;
    T.sub_y0[s] = (double)cy / T.nsy;
    T.sub_hx[s] = 1.0 / ((double)T.nsx * nx);
    T.sub_hy[s] = 1.0 / ((double)T.nsy * ny);
    T.sub_I0[s] = k * cxs[cx]; T.sub_J0[s] = k * cys[cy];
    T.sub_i0[s] = cxs[cx]; T.sub_j0[s] = cys[cy];
  }
  build_templates(T.tpl);
  // offsets
  T.vec_off.assign(S + 1, 0); T.fac_off.assign(S + 1, 0); T.csr_off.assign(S + 1, 0);
  T.unode_off.assign(S + 1, 0); T.pnode_off.assign(S + 1, 0); T.elem_off.assign(S + 1, 0);
  T.sell_off.assign(S + 1, 0);
  for (int s = 0; s < S; ++s) {
    const Template &t = T.tpl[T.sub_tpl[s]];
    T.vec_off[s + 1] = T.vec_off[s] + round_up(t.n, 32);
    T.fac_off[s + 1] = T.fac_off[s] + (long long)t.n * t.LD;
    T.csr_off[s + 1] = T.csr_off[s] + (long long)t.csr_col.size();
    T.unode_off[s + 1] = T.unode_off[s] + (long long)t.nux * t.nuy;
    T.pnode_off[s + 1] = T.pnode_off[s] + (long long)t.npx * t.npy;
    T.elem_off[s + 1] = T.elem_off[s] + 2LL * t.nx * t.ny;
    T.sell_off[s + 1] = T.sell_off[s] + (long long)t.sell_col.size();
  }
  // ---- interface constraints (signed Boolean jump operator, non-redundant chains) ----
  std::map<std::pair<int, int>, std::vector<NodeEnt>> umap, pmap;  // key (J, I) for sorting
  for (int s = 0; s < S; ++s) {
    const Template &t = T.tpl[T.sub_tpl[s]];
    for (int J = 0; J < t.nuy; ++J)
      for (int I = 0; I < t.nux; ++I) {
        if (!(I == 0 || J == 0 || I == t.nux - 1 || J == t.nuy - 1)) continue;
        const int a = J * t.nux + I;
        umap[{T.sub_J0[s] + J, T.sub_I0[s] + I}].push_back({s, t.udof[2 * a], t.udof[2 * a + 1]});
      }
    if (t.poro)
      for (int j = 0; j < t.npy; ++j)
        for (int i = 0; i < t.npx; ++i) {
          if (!(i == 0 || j == 0 || i == t.npx - 1 || j == t.npy - 1)) continue;
          const int b = j * t.npx + i;
          pmap[{T.sub_j0[s] + j, T.sub_i0[s] + i}].push_back({s, t.pdof[b], -1});
        }
  }
  T.lam_key.clear(); T.lam_sa.clear(); T.lam_da.clear(); T.lam_sb.clear(); T.lam_db.clear();
  T.wgrp_first.clear(); T.wgrp_size.clear();
  auto add_rows = [&](int kind, int comp, int I, int J, std::vector<NodeEnt> &ent, int which) {
    const int first = (int)T.lam_sa.size();
    for (size_t q = 0; q + 1 < ent.size(); ++q) {
      const int sa = ent[q].s, sb = ent[q + 1].s;
      const int da = which == 0 ? ent[q].d0 : ent[q].d1;
      const int db = which == 0 ? ent[q + 1].d0 : ent[q + 1].d1;
      T.lam_key.insert(T.lam_key.end(), {kind, comp, I, J, sa, sb});
      T.lam_sa.push_back(sa); T.lam_da.push_back(da);
      T.lam_sb.push_back(sb); T.lam_db.push_back(db);
    }
    const int cnt = (int)T.lam_sa.size() - first;
    if (cnt > 3) return false;
    if (cnt) { T.wgrp_first.push_back(first); T.wgrp_size.push_back(cnt); }
    return true;
  };
  for (auto &kv : umap) {
    auto &ent = kv.second;
    if (ent.size() < 2) continue;
    std::sort(ent.begin(), ent.end(), [](const NodeEnt &a, const NodeEnt &b) { return a.s < b.s; });
    for (int c = 0; c < 2; ++c) {
      bool dir = false;
      for (auto &e : ent) if ((c == 0 ? e.d0 : e.d1) < 0) dir = true;
      if (dir) continue;
      if (!add_rows(0, c, kv.first.second, kv.first.first, ent, c)) { err = "node shared by >4 subdomains"; return false; }
    }
  }
  const int nlu = (int)T.lam_sa.size();
  for (auto &kv : pmap) {
    auto &ent = kv.second;
    if (ent.size() < 2) continue;
    std::sort(ent.begin(), ent.end(), [](const NodeEnt &a, const NodeEnt &b) { return a.s < b.s; });
    bool dir = false;
    for (auto &e : ent) if (e.d0 < 0) dir = true;
    if (dir) continue;
    if (!add_rows(1, 0, kv.first.second, kv.first.first, ent, 0)) { err = "node shared by >4 subdomains"; return false; }
  }
  // device indexing of multiplier arrays (up to 6 entries per row) stays in int
  if (T.lam_sa.size() > (size_t)(INT_MAX / 8)) { err = "too many interface multipliers"; return false; }
  T.n_lambda = (int)T.lam_sa.size();
  T.n_lambda_p = T.n_lambda - nlu;
  // ---- per-subdomain boundary scatter lists ----
  T.bsc_off.assign(S + 1, 0);
  for (int s = 0; s < S; ++s) T.bsc_off[s + 1] = T.bsc_off[s] + (long long)T.tpl[T.sub_tpl[s]].bnd.size();
  T.bsc_row.assign(3 * T.bsc_off[S], -1);
  T.bsc_sign.assign(3 * T.bsc_off[S], 0);
  std::vector<std::vector<int>> bidx(T.tpl.size());
  for (size_t ti = 0; ti < T.tpl.size(); ++ti) {
    bidx[ti].assign(T.tpl[ti].n, -1);
    for (size_t q = 0; q < T.tpl[ti].bnd.size(); ++q) bidx[ti][T.tpl[ti].bnd[q]] = (int)q;
  }
  auto push = [&](int s, int d, int r, int sg) {
    const int q = bidx[T.sub_tpl[s]][d];
    if (q < 0) return false;
    long long base = 3 * (T.bsc_off[s] + q);
    for (int z = 0; z < 3; ++z)
      if (T.bsc_row[base + z] < 0) { T.bsc_row[base + z] = r; T.bsc_sign[base + z] = (int8_t)sg; return true; }
    return false;
  };
  for (int r = 0; r < T.n_lambda; ++r) {
    if (!push(T.lam_sa[r], T.lam_da[r], r, 1) || !push(T.lam_sb[r], T.lam_db[r], r, -1)) {
      err = "interface table inconsistent"; return false;
    }
  }
  for (int s = 0; s < S; ++s)
    for (long long q = T.bsc_off[s]; q < T.bsc_off[s + 1]; ++q)
      if (T.bsc_row[3 * q] < 0) { err = "boundary dof without multiplier"; return false; }
  // ---- coarse space ----
  T.sub_float.assign(S, -1);
  T.float_sub.clear();
  for (int s = 0; s < S; ++s)
    if (T.tpl[T.sub_tpl[s]].floating) { T.sub_float[s] = (int)T.float_sub.size(); T.float_sub.push_back(s); }
  T.NF = (int)T.float_sub.size();
  T.float_rows_ptr.assign(T.NF + 1, 0);
  T.float_rows.clear();
  for (int f = 0; f < T.NF; ++f) {
    const int s = T.float_sub[f];
    std::vector<int> rows;
    for (long long q = T.bsc_off[s]; q < T.bsc_off[s + 1]; ++q)
      for (int z = 0; z < 3; ++z)
        if (T.bsc_row[3 * q + z] >= 0) rows.push_back(T.bsc_row[3 * q + z]);
    std::sort(rows.begin(), rows.end());
    T.float_rows.insert(T.float_rows.end(), rows.begin(), rows.end());
    T.float_rows_ptr[f + 1] = (int)T.float_rows.size();
  }
  T.nH = 3 * T.NF;
  int bf = 0;
  for (int r = 0; r < T.n_lambda; ++r) {
    const int fa = T.sub_float[T.lam_sa[r]], fb = T.sub_float[T.lam_sb[r]];
    if (fa >= 0 && fb >= 0) bf = std::max(bf, std::abs(fa - fb));
  }
  T.bH = T.NF ? 3 * bf + 2 : 0;
  T.LDH = T.NF ? round_up(T.bH + 1, 32) : 0;
  // ---- point source ----
  T.src_sub = -1; T.src_node = -1;
  if (p->source == FP_SOURCE_POINT) {
    for (int s = 0; s < S; ++s) {
      const Template &t = T.tpl[T.sub_tpl[s]];
      const int li = p->src_i - T.sub_i0[s], lj = p->src_j - T.sub_j0[s];
      if (t.poro && li > 0 && li < t.npx - 1 && lj > 0 && lj < t.npy - 1) {
        T.src_sub = s; T.src_node = lj * t.npx + li;
      }
    }
    if (T.src_sub < 0) { err = "point source must lie strictly inside a poroelastic subdomain"; return false; }
  } else if (p->source != FP_SOURCE_MANUFACTURED && p->source != FP_SOURCE_MANUFACTURED_T) {
    err = "unknown source kind"; return false;
  }
  return true;
}

}  // namespace fp
