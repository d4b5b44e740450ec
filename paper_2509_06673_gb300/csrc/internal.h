// Internal data structures of the fetipe library (host and device).
#pragma once
#include <cstdint>
#include <string>
#include <vector>
#include <map>
#include <cuda_runtime.h>

#include "../../include/fetipe.h"

namespace fp {

// Dof fields of the 3-field local system (u, xi, p).
enum Field { F_UX = 0, F_UY = 1, F_XI = 2, F_P = 3 };

// Per-side boundary kind of a subdomain.
enum SideU { SU_CLAMPED = 0, SU_IFACE = 1 };
enum SideP { SP_DIRICHLET = 0, SP_IFACE = 1, SP_NATURAL = 2 };

// A subdomain template: everything that depends only on (nx, ny, k, poro, side kinds).
struct Template {
  int nx, ny, k, poro;
  int side_u[4];  // 0 left, 1 right, 2 bottom, 3 top
  int side_p[4];
  int nux, nuy, npx, npy;
  int transposed;           // band rows run along x (0) or along y (1)
  int n;                    // local dofs
  int b;                    // half bandwidth
  int LD;                   // column stride of the cyclic band layout (multiple of 32, > b)
  int floating;             // no clamped side
  int fixed[3];             // dofs fixed for the generalised inverse (floating only)
  std::vector<int> udof;    // [2 * nux * nuy] dof or -1
  std::vector<int> xidof;   // [npx * npy]
  std::vector<int> pdof;    // [npx * npy] dof or -1
  std::vector<int> dof_field, dof_node;  // [n]
  std::vector<int> csr_ptr, csr_col;     // full symmetric pattern, rows sorted
  std::vector<int> bnd;                  // dofs touched by B_s (sorted)
  std::vector<uint8_t> is_bnd;           // [n]
  // halo rows: rows not in bnd with at least one column in bnd; entries = csr indices
  std::vector<int> halo_ptr, halo_row, halo_ent;
  std::vector<int> elem_dofs;            // [n_elem * ndl] element dof lists (-1 Dirichlet)
  // sliced ELL copy of the Neumann matrix with the generalised-inverse convention (entries in
  // fixed columns dropped, unit diagonal on fixed rows): slices of 32 rows, entry k of row
  // 32 q + l at slot sell_ptr[q] + 32 k + l; sell_src = CSR entry index, -1 padding, -2 unit
  std::vector<int> sell_ptr, sell_col, sell_src;
  int ndl;                               // local dofs per element
};

struct Topology {
  // partition
  int nsx, nsy, poro_rows, k, S;
  std::vector<int> cells_x, cells_y;
  std::vector<Template> tpl;
  std::vector<int> sub_tpl;              // [S]
  std::vector<double> sub_x0, sub_y0, sub_hx, sub_hy;
  std::vector<int> sub_I0, sub_J0, sub_i0, sub_j0;
  std::vector<long long> vec_off;        // [S+1] offsets of local dof vectors
  std::vector<long long> fac_off;        // [S+1] offsets of band factors (elements)
  std::vector<long long> csr_off;        // [S+1] offsets of CSR value arrays
  std::vector<long long> unode_off, pnode_off;  // [S+1] canonical field offsets
  std::vector<long long> elem_off;       // [S+1] element offsets (perm)
  std::vector<long long> sell_off;       // [S+1] offsets of sliced-ELL value arrays
  // interface
  int n_lambda = 0, n_lambda_p = 0;
  std::vector<int> lam_key;              // [6 * n_lambda]
  std::vector<int> lam_sa, lam_da, lam_sb, lam_db;  // [n_lambda]
  // W = (B B^T)^{-1}: groups of consecutive rows of one node component
  std::vector<int> wgrp_first, wgrp_size;
  // per subdomain boundary scatter lists: for bnd dof j of s: rows touching it
  std::vector<long long> bsc_off;        // [S+1] offsets into bnd-entry arrays
  std::vector<int> bsc_row;              // [3 * total_bnd] (-1 pad)
  std::vector<int8_t> bsc_sign;          // [3 * total_bnd]
  // coarse
  int NF = 0;                            // floating subdomains
  std::vector<int> sub_float;            // [S] floating index or -1
  std::vector<int> float_sub;            // [NF]
  std::vector<int> float_rows_ptr, float_rows;   // rows touching each floating subdomain
  int nH = 0, bH = 0, LDH = 0;           // coarse band system
  // point source
  int src_sub = -1, src_node = -1;
};

bool build_topology(const fp_mesh_desc *m, const fp_params *p, Topology &T, std::string &err);

}  // namespace fp
