"""Pins of the oracle's monolithic solution: convergence orders (Tables 3 and 4), the
eta reduction of Sec. 2.5, the interface multiplier against Eq. (2.27), and the
Barry-Mercer no-oscillation property of Sec. 4.3."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.monolithic import Discretization, solve_monolithic
from oracle.errors import linf_l2
from oracle.problem import Manufactured, kappas, lame_from_young
from paper_2509_06673_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table3_p2_orders.txt")


def _errors(k, N, **kw):
    c = W.grid_case("conv", 1, 2, N, N // 2, order_k=k, **kw)
    d = Discretization(c)
    return linf_l2(c, d, solve_monolithic(c, d)), c, d


@pytest.mark.parametrize("k,umin,pmin", [(1, 1.85, 1.75), (2, 2.75, 1.85)])
def test_convergence_orders(k, umin, pmin):
    e = [_errors(k, N, tau=0.01, n_steps=2)[0] for N in (8, 16, 32)]
    ou = np.log2(e[1][0] / e[2][0])
    op = np.log2(e[1][1] / e[2][1])
    assert ou > umin and op > pmin, (ou, op)
    assert ou < k + 1.3 and op < 2.6


def test_golden_table3_p2_orders():
    """Orders of the P2 displacement error, 1/8 -> 1/16, with the paper's parameters."""
    rows = np.loadtxt(GOLD)
    for nu, order in rows:
        lam, mu = lame_from_young(1e4, nu, "paper")
        kw = dict(lame_lambda=lam, mu=mu, c0=0.1, tau=1e-4, n_steps=100)
        e8 = _errors(2, 8, **kw)[0]
        e16 = _errors(2, 16, **kw)[0]
        ours = np.log2(e8[0] / e16[0])
        assert abs(ours - order) < 0.3, (nu, ours, order)


def test_eta_reduction_exact():
    """With W_h = M_h^P the eta row gives eta = (p - k1 xi) / k2 at every node."""
    c = W.small_case(2, 2, 4, k=2, lame_lambda=3.0, alpha=0.7, c0=0.4, tau=0.01, n_steps=2)
    d = Discretization(c)
    st = solve_monolithic(c, d)
    k1, k2, _ = kappas(c.alpha, c.c0, c.lame_lambda)
    for s, L in enumerate(d.locals):
        if L.m.is_poro:
            u, xi, eta, p = st[-1]["fields"][s]
            assert np.abs(eta - (p - k1 * xi) / k2).max() < 1e-10 * (1 + np.abs(eta).max())


@pytest.mark.parametrize("k", [1, 2])
def test_interface_multiplier_converges_to_traction(k):
    """lambda_h = M_Gamma^{-1} lambda_nodal tends to sigma_E(u_E) n_{E->P} (Eq. (2.27))."""
    errs = []
    for N in (8, 16, 32):
        c = W.grid_case("lam", 1, 2, N, N // 2, order_k=k, tau=1e6, n_steps=1)
        d = Discretization(c)
        lam = solve_monolithic(c, d)[-1]["lambda"]
        I = d.iface
        mf = Manufactured(c.lame_lambda, c.mu, c.alpha, c.c0)
        nI = k * N
        # 1D mass matrix of the P_k trace on y = 1/2 over the interior nodes
        h = 1.0 / N
        M = sp.lil_matrix((nI + 1, nI + 1))
        Me = (h / 6) * np.array([[2, 1], [1, 2]]) if k == 1 else \
            (h / 30) * np.array([[4, 2, -1], [2, 16, 2], [-1, 2, 4]])
        for e in range(N):
            idx = [e, e + 1] if k == 1 else [2 * e, 2 * e + 1, 2 * e + 2]
            for a, ia in enumerate(idx):
                for b, ib in enumerate(idx):
                    M[ia, ib] += Me[a, b]
        M = M.tocsr()[1:nI, 1:nI]
        xs = np.arange(1, nI) / nI
        err = 0.0
        for comp in (0, 1):
            nod = np.zeros(nI - 1)
            for r, key in enumerate(I.keys):
                if key[0] == 0 and key[1] == comp:
                    nod[key[2] - 1] = lam[r]
            coef = sp.linalg.spsolve(M.tocsc(), nod)
            ex = mf.traction_on_interface(xs)[comp]
            err += h * np.sum((coef - ex) ** 2)
        errs.append(np.sqrt(err))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders[-1] > 0.9 and errs[-1] < errs[0], (errs, orders)


def test_barry_mercer_no_oscillation():
    """Sec. 4.3: no pressure oscillation at steps 1..3 (tau = 1e-2, T = 1 scale)."""
    lam, mu = lame_from_young(1e4, 0.2)
    for k in (1, 2):
        for N in (16, 32):
            c = W.grid_case("bm", 1, 2, N, N // 2, order_k=k, lame_lambda=lam, mu=mu, c0=0.1,
                            tau=1e-2, n_steps=3, source="barry_mercer", bc="barry_mercer")
            d = Discretization(c)
            for st in solve_monolithic(c, d):
                p = st["fields"][0][3]
                assert p.min() >= -1e-9 * np.abs(p).max()


@pytest.mark.parametrize("k,umin,pmin", [(1, 1.85, 1.75), (2, 2.75, 1.85)])
def test_time_dependent_variant_orders(k, umin, pmin):
    """Closed form times (1 + t): backward Euler is exact in time, so the spatial orders of
    the stationary case are kept."""
    e = []
    for N in (8, 16, 32):
        c = W.grid_case("t", 1, 2, N, N // 2, order_k=k, tau=0.05, n_steps=3, source="manufactured_t")
        d = Discretization(c)
        e.append(linf_l2(c, d, solve_monolithic(c, d)))
    assert np.log2(e[1][0] / e[2][0]) > umin and np.log2(e[1][1] / e[2][1]) > pmin
