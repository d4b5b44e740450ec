"""Monolithic solve of the fully discrete system (test infrastructure; see ``oracle/__init__``).

Per backward-Euler step (Problem 2.4, matrix form Eq. (2.43)) the saddle system

    [ blockdiag(K_s)  B^T ] [ x ]   [ f^n ]
    [ B               0   ] [ l ] = [ 0   ]

is factored once by sparse LU (SuperLU through scipy) and solved for every step; for the
two-subdomain case this is Eq. (2.43) with its rows grouped per subdomain.  Theorem 3.1
gives unique solvability.  Each solve is followed by classical iterative refinement in FP64
(residual b - M x, correction from the same LU factors) until the correction is below
1e-15 of the solution, at most 4 sweeps: the LU solution alone of a nearly incompressible
case (lambda = 499) is off the exact discrete solution by ~1e-10 relative, a refined one by
~1e-16, so the oracle is the block system's solution to rounding.  eta^{n-1} enters through
R eta^{n-1} (Eq. (2.42)); eta^0 is the L2 projection of eta_0, so R eta^0 = (eta_0, phi_i).

Pinned by the convergence-order, transmission and patch tests in tests/test_oracle_*.py, and by
the residual of the block system (tests/test_oracle_feti.py).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .mesh import build_meshes
from .local import LocalSystem
from .jump import Interface


class Discretization:
    """Meshes, local systems and the interface of one case (shared by both solvers)."""

    def __init__(self, case):
        self.case = case
        self.meshes = build_meshes(case)
        self.locals = [LocalSystem(case, m) for m in self.meshes]
        self.iface = Interface(case, self.meshes, self.locals)

    def initial_Reta(self):
        return [L.Reta0() if L.m.is_poro else None for L in self.locals]


def solve_monolithic(case, disc=None, n_steps=None, callback=None, initial=None):
    """Run the time loop; returns a list of per-step dicts with 'lambda' and 'fields'.
    initial: optional per-subdomain (u0, p0) nodal fields (p0 None on elastic subdomains)
    that replace the configured initial state (R eta^0 from eta_0 = c0 p0 + alpha div u0)."""
    disc = disc or Discretization(case)
    Ls, I = disc.locals, disc.iface
    K = sp.block_diag([L.K for L in Ls], format="csr")
    B = sp.hstack(I.Bs, format="csr")
    M = sp.bmat([[K, B.T], [B, None]], format="csc")
    lu = spla.splu(M)

    def solve(rhs):
        x = lu.solve(rhs)
        for _ in range(4):
            dx = lu.solve(rhs - M @ x)
            x = x + dx
            if np.abs(dx).max() <= 1e-15 * np.abs(x).max():
                break
        return x

    offs = np.cumsum([0] + [L.n for L in Ls])
    Reta = disc.initial_Reta()
    if initial is not None:
        Reta = [L.Reta_from_fields(*initial[s]) if L.m.is_poro else None for s, L in enumerate(Ls)]
    out = []
    N = case.n_steps if n_steps is None else n_steps
    for n in range(1, N + 1):
        t = n * case.tau
        rhs = np.concatenate([L.rhs(t, Reta[s]) for s, L in enumerate(Ls)] + [np.zeros(I.n_lambda)])
        x = solve(rhs)
        fields = []
        for s, L in enumerate(Ls):
            fs = L.unpack(x[offs[s]: offs[s + 1]], t)
            fields.append(fs)
            if L.m.is_poro:
                Reta[s] = L.Reta_of(fs[2])
        step = {"n": n, "t": t, "lambda": x[offs[-1]:].copy(), "fields": fields,
                "x": [x[offs[s]: offs[s + 1]].copy() for s in range(len(Ls))]}
        out.append(step)
        if callback:
            callback(step)
    return out
