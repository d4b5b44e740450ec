"""Interface constraints and coarse data (test infrastructure; see ``oracle/__init__``).

The paper couples one poroelastic and one elastic subdomain through
H_P u_P - H_E u_E = 0 (last block row of Eq. (2.43)).  For a grid of subdomains the
project reads it as a signed Boolean jump operator B (the classical FETI choice for the
multiplier space, which the paper leaves unspecified in Sec. 2.4):

* one multiplier per displacement component at every node shared by two or more
  subdomains that is not a displacement Dirichlet node;
* one multiplier for the pressure at every P1 node shared by two or more poroelastic
  subdomains that is not a pressure Dirichlet node (the P-E interface keeps the no-flux
  condition (2.14) as a natural condition);
* at a node shared by subdomains s_1 < s_2 < ... < s_m (ids), the m-1 rows
  x_{s_i} - x_{s_{i+1}} = 0 (non-redundant, so B has full row rank and lambda is unique).
  For the two-subdomain case this is exactly [H_P, -H_E] of Sec. 2.5.

Each row carries a key (kind, comp, I, J, s_a, s_b): kind 0 displacement (comp 0/1, (I, J)
on the global displacement grid), kind 1 pressure (comp 0, (I, J) on the global P1 grid).

Rigid modes of floating subdomains (no displacement Dirichlet node) give the FETI-1 coarse
space G = [B_s R_s] (not in the paper, which has no floating subdomain).

Pinned by tests/test_oracle_feti.py (B full row rank, B applied to a continuous field is
zero, K_s R_s = 0, the FETI solution equals the monolithic one).
"""
import numpy as np
import scipy.sparse as sp


class Interface:
    def __init__(self, case, meshes, locals_):
        self.case = case
        self.nsub = len(meshes)
        umap, pmap = {}, {}
        for m, L in zip(meshes, locals_):
            inv_u = -np.ones(2 * m.n_unode, dtype=np.int64)
            inv_u[L.ufree] = np.arange(L.ufree.size)
            for a in range(m.n_unode):
                key = m.unode_key(a)
                umap.setdefault(key, []).append((m.s, a, inv_u[2 * a], inv_u[2 * a + 1]))
            if m.is_poro:
                inv_p = -np.ones(m.n_pnode, dtype=np.int64)
                inv_p[L.pfree] = np.arange(L.pfree.size)
                for b in range(m.n_pnode):
                    key = m.pnode_key(b)
                    pmap.setdefault(key, []).append((m.s, b, inv_p[b]))
        rows = []  # (key, [(s, local_dof, sign)])
        for key in sorted(umap, key=lambda k: (k[1], k[0])):
            ent = sorted(umap[key])
            if len(ent) < 2:
                continue
            for c in (0, 1):
                if any(e[2 + c] < 0 for e in ent):
                    continue  # Dirichlet component
                for i in range(len(ent) - 1):
                    sa, sb = ent[i][0], ent[i + 1][0]
                    rows.append(((0, c, key[0], key[1], sa, sb),
                                 [(sa, ent[i][2 + c], 1.0), (sb, ent[i + 1][2 + c], -1.0)]))
        for key in sorted(pmap, key=lambda k: (k[1], k[0])):
            ent = sorted(pmap[key])
            if len(ent) < 2 or any(e[2] < 0 for e in ent):
                continue
            for i in range(len(ent) - 1):
                sa, sb = ent[i][0], ent[i + 1][0]
                La, Lb = locals_[sa], locals_[sb]
                rows.append(((1, 0, key[0], key[1], sa, sb),
                             [(sa, La.off_p + ent[i][2], 1.0), (sb, Lb.off_p + ent[i + 1][2], -1.0)]))
        self.keys = [r[0] for r in rows]
        self.n_lambda = len(rows)
        self.is_p = np.array([k[0] == 1 for k in self.keys], dtype=bool)
        trip = [[] for _ in range(self.nsub)]
        for r, (_, ents) in enumerate(rows):
            for s, d, sg in ents:
                trip[s].append((r, d, sg))
        self.Bs = []
        for s, L in enumerate(locals_):
            if trip[s]:
                r, d, v = zip(*trip[s])
            else:
                r, d, v = (), (), ()
            self.Bs.append(sp.csr_matrix((v, (r, d)), shape=(self.n_lambda, L.n)))
        self._scaling()
        self._coarse(meshes, locals_)

    def _scaling(self):
        """W = (B B^T)^{-1}: block diagonal with one small block per (node, field comp)."""
        BBt = sum((B @ B.T) for B in self.Bs).tocsc()
        self.BBt = BBt
        self.W = sp.csc_matrix(np.linalg.inv(BBt.toarray())) if self.n_lambda < 4000 else None
        if self.W is None:
            import scipy.sparse.linalg as spla
            lu = spla.splu(BBt)
            self._W_lu = lu

    def apply_W(self, v):
        if self.W is not None:
            return self.W @ v
        return self._W_lu.solve(v)

    def _coarse(self, meshes, locals_):
        self.floating = []
        self.Rs = [None] * self.nsub
        self.fixed = [None] * self.nsub
        for m, L in zip(meshes, locals_):
            if L.du.any():
                continue
            self.floating.append(m.s)
            x, y = m.unode_xy()
            xc, yc = 0.5 * (m.x0 + m.x1), 0.5 * (m.y0 + m.y1)
            size = max(m.x1 - m.x0, m.y1 - m.y0)
            R = np.zeros((L.n, 3))
            R[0: L.nu: 2, 0] = 1.0
            R[1: L.nu: 2, 1] = 1.0
            R[0: L.nu: 2, 2] = -(y - yc) / size
            R[1: L.nu: 2, 2] = (x - xc) / size
            self.Rs[m.s] = R
            # three fixed dofs that block the rigid motions: node (0,0) x and y, node
            # (k*nx, 0) y  (all dofs are free on a floating subdomain)
            a_far = m.nux - 1
            self.fixed[m.s] = np.array([0, 1, 2 * a_far + 1])
        cols = [self.Bs[s] @ self.Rs[s] for s in self.floating]
        self.G = np.hstack(cols) if cols else np.zeros((self.n_lambda, 0))
        self.GtG = self.G.T @ self.G

    def e_vector(self, f_list):
        return np.concatenate([self.Rs[s].T @ f_list[s] for s in self.floating]) \
            if self.floating else np.zeros(0)
