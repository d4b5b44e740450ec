"""FETI solve of the interface problem (test infrastructure; see ``oracle/__init__``).

Sec. 3.1 reduces each step to K_S lambda = F_S (Eq. (3.3)) with
K_S = sum_s H_s S_s^{-1} H_s^T, and Sec. 3.2 shows the same operator is
K_A = sum_s H_s K_s^{-1} H_s^T (Eq. (3.6)), which needs no nested iteration.  With the
Boolean B (see ``jump``):

    F = sum_s B_s K_s^+ B_s^T,   d = sum_s B_s K_s^+ f_s,

where K_s^+ is the inverse of K_s, or for a floating subdomain the generalised inverse that
fixes three displacement dofs.  Floating subdomains add the FETI-1 coarse problem
(G = [B_s R_s], e = [R_s^T f_s], projector P = I - G (G^T G)^{-1} G^T), which the paper's
two-subdomain setting does not need.

Krylov: Algorithm 1 (PCG) with the Dirichlet preconditioner of Eq. (3.5),
M^{-1} = sum_s B_s S_s B_s^T scaled by W = (B B^T)^{-1} on both sides, reading the
misprinted z_{k+1} = M^{-1} z_k as z_{k+1} = M^{-1} r_{k+1}, and starting from
lambda^{n-1} (Algorithm 1's warm start) projected onto the constraint G^T lambda = e.
When pressure multipliers exist (several poroelastic subdomains) F is symmetric
indefinite (its pressure block is negative definite).  The Dirichlet preconditioner then
has the same inertia as F and the preconditioned operator keeps a real spectrum >= 1 on
range(P) (checked in tests/test_oracle_feti.py), so Algorithm 1 is still the default;
breakdown (p^T F p = 0 or non-finite) is reported.  As the textbook alternative for
symmetric indefinite systems the oracle also offers preconditioned MINRES (Paige &
Saunders 1975; not in the paper) with the symmetric positive definite block form
diag(S_uu, -S_pp) of the same preconditioner.  Both stop when
||P(d - F lambda)||_2 <= tol * ||P(d - F lambda_00)||_2, lambda_00 = G (G^T G)^{-1} e
(the paper only says "until convergence").  Recovery (proof of Theorem 3.1):
alpha = (G^T G)^{-1} G^T (F lambda - d), x_s = K_s^+ (f_s - B_s^T lambda) + R_s alpha_s.

Pinned by tests/test_oracle_feti.py: FETI equals the monolithic solution, F symmetric with
the expected inertia, G^T lambda = e, B x = 0, invariance to the fixed dofs, PCG and MINRES
against dense solves.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .monolithic import Discretization


def pcg(apply_A, apply_Minv, b_res, x0, tol, ref, max_it):
    """Algorithm 1 (with z_{k+1} = M^{-1} r_{k+1}) for a symmetric operator.

    ``b_res`` is the initial residual b - A x0 (already projected by the caller's operators).
    Returns x, iterations, history of ||r||_2.
    """
    x = x0.copy()
    r = b_res.copy()
    z = apply_Minv(r)
    p = z.copy()
    rz = r @ z
    hist = [np.linalg.norm(r)]
    k = 0
    while hist[-1] > tol * ref and k < max_it:
        q = apply_A(p)
        pq = p @ q
        if pq == 0.0 or not np.isfinite(pq):
            raise FloatingPointError("PCG breakdown: p^T F p = %r" % pq)
        alpha = rz / pq
        x += alpha * p
        r -= alpha * q
        z = apply_Minv(r)
        rz_new = r @ z
        beta = rz_new / rz
        p = z + beta * p
        rz = rz_new
        k += 1
        hist.append(np.linalg.norm(r))
    return x, k, hist


def minres(apply_A, apply_Minv, b_res, x0, tol, ref, max_it):
    """Preconditioned MINRES (Paige & Saunders 1975) for symmetric indefinite A and SPD M.

    Besides the standard recurrences it carries A w_k so that the true residual
    r_k = b - A x_k is updated explicitly and the 2-norm stop test is exact.
    """
    n = b_res.size
    x = x0.copy()
    r = b_res.copy()                      # tracked true residual
    r1 = b_res.copy()
    r2 = b_res.copy()
    y = apply_Minv(r1)
    beta1 = np.sqrt(max(r1 @ y, 0.0))
    hist = [np.linalg.norm(r)]
    if beta1 == 0.0:
        return x, 0, hist
    oldb, beta, dbar, epsln, phibar = 0.0, beta1, 0.0, 0.0, beta1
    cs, sn = -1.0, 0.0
    w = np.zeros(n); w2 = np.zeros(n)
    Aw = np.zeros(n); Aw2 = np.zeros(n)
    k = 0
    while hist[-1] > tol * ref and k < max_it:
        v = y / beta
        Av = apply_A(v)
        y = Av.copy()
        if k > 0:
            y -= (beta / oldb) * r1
        alfa = v @ y
        y -= (alfa / beta) * r2
        r1, r2 = r2, y
        y = apply_Minv(r2)
        oldb = beta
        beta = np.sqrt(max(r2 @ y, 0.0))
        oldeps = epsln
        delta = cs * dbar + sn * alfa
        gbar = sn * dbar - cs * alfa
        epsln = sn * beta
        dbar = -cs * beta
        gamma = np.hypot(gbar, beta)
        cs, sn = gbar / gamma, beta / gamma
        phi = cs * phibar
        phibar = sn * phibar
        w1, w2 = w2, w
        Aw1, Aw2 = Aw2, Aw
        w = (v - oldeps * w1 - delta * w2) / gamma
        Aw = (Av - oldeps * Aw1 - delta * Aw2) / gamma
        x += phi * w
        r -= phi * Aw
        k += 1
        hist.append(np.linalg.norm(r))
        if beta == 0.0:
            break
    return x, k, hist


class FETI:
    def __init__(self, case, disc=None, fixed_override=None, precond=None):
        self.case = case
        # "dirichlet" (Eq. (3.5)), "lumped" (Sec. 3.3: the M_A of Algorithm 2, which reduces to
        # the local matrices' interface block K_bb) or "none"
        self.precond_kind = precond or getattr(case, "precond", "dirichlet")
        if self.precond_kind not in ("dirichlet", "lumped", "none"):
            self.precond_kind = "dirichlet"
        self.disc = disc or Discretization(case)
        Ls, I = self.disc.locals, self.disc.iface
        self.Ls, self.I = Ls, I
        self.has_p = bool(I.is_p.any())
        # Neumann (generalised) inverses ----------------------------------------------
        self.keep, self.lu = [], []
        for s, L in enumerate(Ls):
            fixed = I.fixed[s]
            if fixed_override is not None and fixed is not None:
                fixed = fixed_override(s, L)
            keep = np.arange(L.n) if fixed is None else np.setdiff1d(np.arange(L.n), fixed)
            self.keep.append(keep)
            self.lu.append(spla.splu(L.K[keep][:, keep].tocsc()))
        # Dirichlet data ---------------------------------------------------------------
        self.bd, self.bu_mask, self.dlu, self.Kbb, self.Kbi, self.Kib = [], [], [], [], [], []
        self.Kbb3 = []
        for s, L in enumerate(Ls):
            Bs = I.Bs[s].tocsc()
            bd = np.flatnonzero(np.diff(Bs.indptr))
            idof = np.setdiff1d(np.arange(L.n), bd)
            K = L.K.tocsr()
            self.bd.append(bd)
            is_pdof = bd >= L.off_p if L.m.is_poro else np.zeros(bd.size, dtype=bool)
            self.bu_mask.append(~is_pdof)
            self.dlu.append(spla.splu(K[idof][:, idof].tocsc()) if bd.size else None)
            self.Kbb.append(K[bd][:, bd])
            self.Kbi.append(K[bd][:, idof])
            self.Kib.append(K[idof][:, bd])
            # interface block of the 3-field local matrix (eta eliminated, the library's local
            # system): the 4-field K_bb plus -(c0 + alpha^2 / lambda) R on the pressure dofs
            Kb3 = K[bd][:, bd].toarray()
            if L.m.is_poro and is_pdof.any():
                ip = np.flatnonzero(is_pdof)
                nodes = L.pfree[bd[ip] - L.off_p]
                c = case.c0 + case.alpha ** 2 / case.lame_lambda
                Kb3[np.ix_(ip, ip)] -= c * L.R_full[nodes][:, nodes].toarray()
            self.Kbb3.append(Kb3)
        # coarse -----------------------------------------------------------------------
        self.nc = I.G.shape[1]
        self.GtG_cho = sla.cho_factor(I.GtG) if self.nc else None

    # operators --------------------------------------------------------------------------
    def Kplus(self, s, b):
        x = np.zeros_like(b)
        keep = self.keep[s]
        x[keep] = self.lu[s].solve(b[keep])
        return x

    def F(self, v):
        out = np.zeros(self.I.n_lambda)
        for s, B in enumerate(self.I.Bs):
            out += B @ self.Kplus(s, B.T @ v)
        return out

    def S_apply(self, s, xb):
        """Dirichlet Schur complement S_s = K_bb - K_bi K_ii^{-1} K_ib on boundary dofs."""
        y = self.Kbb[s] @ xb
        if self.dlu[s] is not None and self.Kib[s].shape[0]:
            y -= self.Kbi[s] @ self.dlu[s].solve(self.Kib[s] @ xb)
        return y

    def local_precond(self, s, xb):
        """The local operator of the preconditioner on the interface dofs of s: the Dirichlet
        Schur complement S_s, or the lumped interface block K_bb of the 3-field matrix."""
        if self.precond_kind == "lumped":
            return self.Kbb3[s] @ xb
        return self.S_apply(s, xb)

    def precond(self, r, block=False):
        """W sum_s B_s S^_s B_s^T W r with S^_s = S_s (Eq. (3.5); K_bb for the lumped
        preconditioner), or with ``block`` the positive definite diag(S_uu, -S_pp) used by
        MINRES.  The identity for precond "none"."""
        if self.precond_kind == "none":
            return np.array(r, dtype=np.float64)
        I = self.I
        rw = I.apply_W(r)
        out = np.zeros(I.n_lambda)
        for s, B in enumerate(I.Bs):
            bd = self.bd[s]
            if bd.size == 0:
                continue
            yb = (B.T @ rw)[bd]
            um = self.bu_mask[s]
            if block and (~um).any():
                zu = self.local_precond(s, np.where(um, yb, 0.0))
                zp = self.local_precond(s, np.where(um, 0.0, yb))
                zb = np.where(um, zu, -zp)
            else:
                zb = self.local_precond(s, yb)
            full = np.zeros(self.Ls[s].n)
            full[bd] = zb
            out += B @ full
        return I.apply_W(out)

    def P(self, v):
        if not self.nc:
            return v
        G = self.I.G
        return v - G @ sla.cho_solve(self.GtG_cho, G.T @ v)

    # one step ---------------------------------------------------------------------------
    def solve_step(self, f_list, lam_guess, tol=None, max_it=None, krylov=None):
        I = self.I
        tol = self.case.tol if tol is None else tol
        max_it = self.case.max_it if max_it is None else max_it
        d = np.zeros(I.n_lambda)
        for s, B in enumerate(I.Bs):
            d += B @ self.Kplus(s, f_list[s])
        if self.nc:
            e = I.e_vector(f_list)
            lam00 = I.G @ sla.cho_solve(self.GtG_cho, e)
        else:
            lam00 = np.zeros(I.n_lambda)
        lam0 = lam00 + self.P(lam_guess)
        ref = np.linalg.norm(self.P(d - self.F(lam00)))
        r0 = self.P(d - self.F(lam0))
        kind = krylov or "pcg"
        A = lambda v: self.P(self.F(v))
        Minv = lambda v: self.P(self.precond(self.P(v), block=(kind == "minres")))
        solver = minres if kind == "minres" else pcg
        if ref == 0.0:
            return lam0, 0, [0.0], d
        dlam, its, hist = solver(A, Minv, r0, np.zeros(I.n_lambda), tol, ref, max_it)
        lam = lam0 + dlam
        return lam, its, [h / ref for h in hist], d

    def recover(self, f_list, lam, d):
        I = self.I
        xs = []
        if self.nc:
            alpha = sla.cho_solve(self.GtG_cho, I.G.T @ (self.F(lam) - d))
        j = 0
        for s, B in enumerate(I.Bs):
            x = self.Kplus(s, f_list[s] - B.T @ lam)
            if I.Rs[s] is not None:
                x += I.Rs[s] @ alpha[3 * j: 3 * j + 3]
                j += 1
            xs.append(x)
        return xs

    def run(self, n_steps=None, lam_init=None, callback=None, krylov=None):
        case, Ls = self.case, self.Ls
        Reta = self.disc.initial_Reta()
        lam = np.zeros(self.I.n_lambda) if lam_init is None else lam_init.copy()
        out = []
        N = case.n_steps if n_steps is None else n_steps
        for n in range(1, N + 1):
            t = n * case.tau
            f = [L.rhs(t, Reta[s]) for s, L in enumerate(Ls)]
            lam, its, hist, d = self.solve_step(f, lam, krylov=krylov)
            xs = self.recover(f, lam, d)
            fields = []
            for s, L in enumerate(Ls):
                fs = L.unpack(xs[s], t)
                fields.append(fs)
                if L.m.is_poro:
                    Reta[s] = L.Reta_of(fs[2])
            step = {"n": n, "t": t, "lambda": lam.copy(), "fields": fields, "x": xs,
                    "iterations": its, "history": hist}
            out.append(step)
            if callback:
                callback(step)
        return out

    # dense helpers for property tests (small cases only) -----------------------------
    def dense_F(self):
        n = self.I.n_lambda
        return np.column_stack([self.F(np.eye(n)[:, j]) for j in range(n)])
