"""L2 errors against the closed-form solution (test infrastructure; see ``oracle/__init__``).

Tables 3 and 4 report L_inf(L2) errors: the maximum over time steps of the L2 error over
Omega (displacement) and Omega^P (pressure).  Integrated with ``collapsed_gauss(6)``
(exact to degree 10).  Pinned by the convergence-order tests.
"""
import numpy as np

from . import fem
from .quadrature import collapsed_gauss
from .problem import Manufactured, time_factor


def l2_errors(case, disc, fields, t=0.0):
    """(||u_h - u||, ||p_h - p||, ||xi_h - xi||, ||eta_h - eta||) for one time level."""
    mf = Manufactured(case.lame_lambda, case.mu, case.alpha, case.c0, case.perm_k, case.mu_f)
    g = time_factor(t)[0] if case.source == "manufactured_t" else 1.0
    lam, w = collapsed_gauss(6)
    eu = ep = ex = ee = 0.0
    for L, fs in zip(disc.locals, fields):
        m = L.m
        u, xi, eta, p = fs
        _, area = fem.bary_grads(m.elem_xy)
        X = fem.map_points(m.elem_xy, lam)
        x, y = X[..., 0], X[..., 1]
        wa = w[None, :] * area[:, None]
        phik = fem.shape(m.k, lam)
        phi1 = fem.shape(1, lam)
        uh = np.einsum("qi,eic->eqc", phik, u[m.elem_u])
        ux, uy = (mf.u_P if m.is_poro else mf.u_E)(x, y)
        ux, uy = g * ux, g * uy
        eu += np.sum(wa * ((uh[..., 0] - ux) ** 2 + (uh[..., 1] - uy) ** 2))
        xih = np.einsum("qi,ei->eq", phi1, xi[m.elem_p])
        xie = g * (mf.xi_P if m.is_poro else mf.xi_E)(x, y)
        ex += np.sum(wa * (xih - xie) ** 2)
        if m.is_poro:
            ph = np.einsum("qi,ei->eq", phi1, p[m.elem_p])
            ep += np.sum(wa * (ph - g * mf.p(x, y)) ** 2)
            eh = np.einsum("qi,ei->eq", phi1, eta[m.elem_p])
            ee += np.sum(wa * (eh - g * mf.eta(x, y)) ** 2)
    return np.sqrt(eu), np.sqrt(ep), np.sqrt(ex), np.sqrt(ee)


def linf_l2(case, disc, steps):
    errs = np.array([l2_errors(case, disc, st["fields"], st["t"]) for st in steps])
    return errs.max(axis=0)
