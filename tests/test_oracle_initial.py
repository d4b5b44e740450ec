"""Pins of the oracle's initial state from given fields, R eta^0 = (c0 p0 + alpha div u0, phi_i)
(Sec. 2.5, Eq. 2.17), against closed-form integrals on the mesh geometry (no use of the
oracle's own mass or divergence matrices): for a linear integrand f the exact P1 load is
int_T f phi_i = |T| (2 f_i + f_j + f_k) / 12 on every triangle T."""
import numpy as np

from oracle.monolithic import Discretization
from paper_2509_06673_gb300 import workloads as W


def _case():
    return W.grid_case("init", 2, 2, [3, 4], [2, 3], order_k=2, lame_lambda=7.0, alpha=0.8, c0=0.3,
                       tau=1e-2)


def _linear_load(m, f):
    """sum over triangles of |T| (2 f_i + f_j + f_k) / 12 for f given at the P1 vertices."""
    out = np.zeros(m.n_pnode)
    xy = np.stack(m.pnode_xy(), axis=1)
    fv = f(xy[:, 0], xy[:, 1])
    for e in range(m.elem_p.shape[0]):
        v = m.elem_p[e]
        P = xy[v]
        area = 0.5 * abs((P[1, 0] - P[0, 0]) * (P[2, 1] - P[0, 1]) - (P[1, 1] - P[0, 1]) * (P[2, 0] - P[0, 0]))
        tot = fv[v].sum()
        for a in range(3):
            out[v[a]] += area * (fv[v[a]] + tot) / 12.0
    return out


def test_initial_from_fields_closed_forms():
    case = _case()
    d = Discretization(case)
    for L in d.locals:
        m = L.m
        if not m.is_poro:
            continue
        ux, uy = m.unode_xy()
        # u0 = (x, 0): div = 1
        u0 = np.stack([ux, 0 * ux], axis=1)
        got = L.Reta_from_fields(u0, None)
        ref = case.alpha * _linear_load(m, lambda x, y: 1.0 + 0 * x)
        assert np.abs(got - ref).max() < 1e-14
        # p0 = 1 + 2x - y (linear, exact in P1)
        px, py = m.pnode_xy()
        got = L.Reta_from_fields(None, 1 + 2 * px - py)
        ref = case.c0 * _linear_load(m, lambda x, y: 1 + 2 * x - y)
        assert np.abs(got - ref).max() < 1e-14
        # u0 = (x y, y^2 / 2) in P2: div = 2 y (linear); plus p0 = x
        u0 = np.stack([ux * uy, 0.5 * uy * uy], axis=1)
        got = L.Reta_from_fields(u0, px)
        ref = _linear_load(m, lambda x, y: case.c0 * x + case.alpha * 2 * y)
        assert np.abs(got - ref).max() < 1e-14
        # partition of unity: the entries of the div-1 load sum to alpha |Omega_s|
        area = (m.x1 - m.x0) * (m.y1 - m.y0)
        assert abs(L.Reta_from_fields(np.stack([ux, 0 * ux], axis=1), None).sum() - case.alpha * area) < 1e-14
