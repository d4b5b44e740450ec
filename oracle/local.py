"""Per-subdomain systems (test infrastructure; see ``oracle/__init__``).

The poroelastic block is the literal 4-field block of the system in Sec. 2.5
(Eq. (2.43)), rows and unknowns (u, xi, eta, p):

    [ A      B^T      0        0     ]
    [ B   -k3 R    k1 R       0     ]
    [ 0    k1 R    k2 R      -R     ]
    [ 0      0      -R     -tau Af  ]

with right-hand side (F_P, 0, 0, -R eta^{n-1} - tau Z) (Eq. (2.42) folded into the
fourth row).  The elastic block is [[A, B^T], [B, -R/lambda]] with (F_E, 0).
Dirichlet values of u (and of p) are eliminated by lifting.  Readings: W_h = M_h^P
(Sec. 2.4), so xi and eta carry every P1 node and only p carries the pressure Dirichlet
condition; the elastic load is f_E (the "f_P" in Eq. (2.38) is a misprint).

Pinned by the convergence-order, patch, eta-reduction and transmission tests
(tests/test_oracle_solution.py, tests/test_oracle_problem.py), the initial-data test
(tests/test_oracle_initial.py), the point-source load and fluid-balance tests
(tests/test_oracle_point_source.py), the dense 3-field comparison and the block-system
residual (tests/test_oracle_feti.py).
"""
import numpy as np
import scipy.sparse as sp

from . import fem
from .problem import Manufactured, kappas, barry_mercer_p2, time_factor


def _dirichlet(case, m):
    """Dirichlet masks for u (n_unode, 2) and p (n_pnode) of subdomain mesh m."""
    Imax = m.k * int(sum(case.cells_x))
    Jmax = m.k * int(sum(case.cells_y))
    imax = int(sum(case.cells_x))
    a = np.arange(m.n_unode)
    I = m.I0 + a % m.nux
    J = m.J0 + a // m.nux
    b = np.arange(m.n_pnode)
    i = m.i0 + b % m.npx
    j = m.j0 + b // m.npx
    du = np.zeros((m.n_unode, 2), dtype=bool)
    dp = np.zeros(m.n_pnode, dtype=bool)
    if case.bc == "clamped":
        on = (I == 0) | (I == Imax) | (J == 0) | (J == Jmax)
        du[:, 0] = on
        du[:, 1] = on
        if m.is_poro:
            dp[:] = (i == 0) | (i == imax) | (j == 0)
    elif case.bc == "barry_mercer":
        du[:, 0] = (I == 0) | (I == Imax)
        du[:, 1] = (J == 0) | (J == Jmax)
        if m.is_poro:
            dp[:] = (i == 0) | (i == imax) | (j == 0)
    else:
        raise ValueError(case.bc)
    return du, dp


def _assemble(n, elem_dofs, Ke):
    ne, nl = elem_dofs.shape
    rows = np.repeat(elem_dofs, nl, axis=1).ravel()
    cols = np.tile(elem_dofs, (1, nl)).ravel()
    return sp.csr_matrix((Ke.ravel(), (rows, cols)), shape=n)


class LocalSystem:
    """Assembled subdomain block with Dirichlet elimination."""

    def __init__(self, case, m):
        self.case, self.m = case, m
        lam, mu, alpha, c0 = case.lame_lambda, case.mu, case.alpha, case.c0
        self.k1, self.k2, self.k3 = kappas(alpha, c0, lam)
        perm = None if case.perm is None else case.perm[m.s]
        if perm is None:
            perm = np.full(2 * m.nx * m.ny, float(case.perm_k))
        Ae, Be, Re, Afe = fem.element_matrices(m.elem_xy, m.k, mu, perm, case.mu_f)
        nl = m.elem_u.shape[1]
        udofs = np.empty((m.elem_u.shape[0], 2 * nl), dtype=np.int64)
        udofs[:, 0::2] = 2 * m.elem_u
        udofs[:, 1::2] = 2 * m.elem_u + 1
        nU, nP = 2 * m.n_unode, m.n_pnode
        self.A_full = _assemble((nU, nU), udofs, Ae)
        ne = udofs.shape[0]
        rows = np.repeat(m.elem_p, 2 * nl, axis=1).ravel()
        cols = np.tile(udofs, (1, 3)).ravel()
        self.B_full = sp.csr_matrix((Be.ravel(), (rows, cols)), shape=(nP, nU))
        self.R_full = _assemble((nP, nP), m.elem_p, Re)
        self.Af_full = _assemble((nP, nP), m.elem_p, Afe)
        assert ne == 2 * m.nx * m.ny

        du, dp = _dirichlet(case, m)
        self.du, self.dp = du, dp
        self.ufree = np.flatnonzero(~du.ravel())            # indices into 2*n_unode
        self.pfree = np.flatnonzero(~dp) if m.is_poro else np.zeros(0, dtype=np.int64)
        self.pdir = np.flatnonzero(dp) if m.is_poro else np.zeros(0, dtype=np.int64)
        nu = self.ufree.size
        self.nu, self.np1 = nu, nP
        A = self.A_full[self.ufree][:, self.ufree]
        B = self.B_full[:, self.ufree]
        R = self.R_full
        if m.is_poro:
            npf = self.pfree.size
            Rp = R[:, self.pfree]
            Z = None
            self.K = sp.bmat([
                [A, B.T, Z, Z],
                [B, -self.k3 * R, self.k1 * R, Z],
                [Z, self.k1 * R, self.k2 * R, -Rp],
                [Z, Z, -Rp.T, -case.tau * self.Af_full[self.pfree][:, self.pfree]],
            ], format="csr")
            self.off_xi, self.off_eta, self.off_p = nu, nu + nP, nu + 2 * nP
            self.n = nu + 2 * nP + npf
        else:
            self.K = sp.bmat([[A, B.T], [B, -R / lam]], format="csr")
            self.off_xi = nu
            self.n = nu + nP
        self._loads()

    # loads ------------------------------------------------------------------------
    def _loads(self):
        case, m = self.case, self.m
        nU, nP = 2 * m.n_unode, m.n_pnode
        nl = m.elem_u.shape[1]
        udofs = np.empty((m.elem_u.shape[0], 2 * nl), dtype=np.int64)
        udofs[:, 0::2] = 2 * m.elem_u
        udofs[:, 1::2] = 2 * m.elem_u + 1
        self.F_full = np.zeros(nU)
        self.Z_full = np.zeros(nP)
        self.eta0_load = np.zeros(nP)
        if case.source in ("manufactured", "manufactured_t"):
            mf = Manufactured(case.lame_lambda, case.mu, case.alpha, case.c0, case.perm_k, case.mu_f)
            f = mf.f_P if m.is_poro else mf.f_E
            np.add.at(self.F_full, udofs, fem.load_vector_u(m.elem_xy, m.k, f))
            if m.is_poro:
                np.add.at(self.Z_full, m.elem_p, fem.load_vector_s(m.elem_xy, mf.z))
                np.add.at(self.eta0_load, m.elem_p, fem.load_vector_s(m.elem_xy, mf.eta))
        # point source and Barry-Mercer: f = 0, z = 0 or a nodal point load, eta_0 = 0

    def point_node(self):
        """Local P1 index of the point source in this subdomain, or -1."""
        case, m = self.case, self.m
        if case.source != "point" or not m.is_poro:
            return -1
        i, j = case.src_node
        li, lj = i - m.i0, j - m.j0
        if 0 <= li < m.npx and 0 <= lj < m.npy:
            return lj * m.npx + li
        return -1

    def p_dirichlet_values(self, t):
        m = self.m
        if self.pdir.size == 0:
            return np.zeros(0)
        if self.case.bc == "barry_mercer":
            x, y = m.pnode_xy()
            x, y = x[self.pdir], y[self.pdir]
            j = m.j0 + self.pdir // m.npx
            return np.where(j == 0, barry_mercer_p2(x, t), 0.0)
        return np.zeros(self.pdir.size)

    def rhs(self, t, Reta_prev):
        """Right-hand side at time t given R eta^{n-1} (full P1 vector)."""
        case = self.case
        b = np.zeros(self.n)
        g, dg = time_factor(t) if case.source == "manufactured_t" else (1.0, 0.0)
        b[: self.nu] = g * self.F_full[self.ufree]
        if self.m.is_poro:
            Z = g * self.Z_full + dg * self.eta0_load
            pn = self.point_node()
            if pn >= 0:
                Z[pn] += np.sin(case.q_omega * t)
            pD = self.p_dirichlet_values(t)
            # eta-row: k1 R xi + k2 R eta - R p = 0 with p = p_free + p_D lifted
            b[self.off_eta: self.off_eta + self.np1] = self.R_full[:, self.pdir] @ pD
            # p-row: -R eta - tau Af p = -R eta^{n-1} - tau Z
            b[self.off_p:] = (-Reta_prev[self.pfree] - case.tau * Z[self.pfree]
                              + case.tau * (self.Af_full[self.pfree][:, self.pdir] @ pD))
        return b

    def Reta_from_fields(self, u0, p0):
        """R eta^0 = (eta_0, phi_i) for eta_0 = c0 p0 + alpha div u0 (Sec. 2.5 with Eq. 2.17) from
        nodal fields: u0 (n_unode, 2) or flat 2 n_unode, p0 (n_pnode,), interpolated in P_k and
        P1 on every node.  B_full = -(phi_i, div theta_j), so (div u0, phi_i) = -(B_full u0)_i."""
        m, case = self.m, self.case
        u = np.zeros(2 * m.n_unode) if u0 is None else np.asarray(u0, dtype=np.float64).ravel()
        p = np.zeros(m.n_pnode) if p0 is None else np.asarray(p0, dtype=np.float64)
        return case.c0 * (self.R_full @ p) - case.alpha * (self.B_full @ u)

    def Reta0(self):
        """R eta^0 for the L2 projection eta^0 of eta_0 (Sec. 2.5): the load (eta_0, phi_i)."""
        return self.eta0_load.copy()

    # unpacking --------------------------------------------------------------------
    def unpack(self, x, t):
        """Local solution -> node arrays (u (n_unode, 2), xi, eta, p) with Dirichlet data."""
        m = self.m
        u = np.zeros(2 * m.n_unode)
        u[self.ufree] = x[: self.nu]
        u = u.reshape(-1, 2)
        xi = x[self.off_xi: self.off_xi + self.np1].copy()
        if m.is_poro:
            eta = x[self.off_eta: self.off_eta + self.np1].copy()
            p = np.zeros(self.np1)
            p[self.pfree] = x[self.off_p:]
            p[self.pdir] = self.p_dirichlet_values(t)
            return u, xi, eta, p
        return u, xi, None, None

    def Reta_of(self, eta):
        return self.R_full @ eta
