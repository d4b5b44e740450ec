"""Pins of the oracle's FETI solve: agreement with the monolithic solution (Theorem 3.1),
operator properties, coarse constraints, Krylov methods against dense solves."""
import numpy as np
import pytest

from oracle.monolithic import Discretization, solve_monolithic
from oracle.feti import FETI, pcg, minres
from paper_2509_06673_gb300 import workloads as W


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _lognormal(case):
    return case.with_(perm=W.lognormal_perm(case, sigma=1.0, seed=0))


@pytest.mark.parametrize("krylov", ["pcg", "minres"])
@pytest.mark.parametrize("case", [
    W.config1(n_steps=3, tol=1e-13),
    W.small_case(4, 4, 3, k=2, lame_lambda=49.0, tau=1e-3, n_steps=2, tol=1e-13),
    W.grid_case("uneven", 3, 4, [2, 4, 3], [3, 2, 4, 3], order_k=1, lame_lambda=5.0,
                c0=0.5, tau=1e-2, n_steps=2, tol=1e-13),
    _lognormal(W.small_case(4, 4, 3, k=2, lame_lambda=499.0, tau=1e-3, n_steps=2, tol=1e-14,
                            source="manufactured_t", max_it=3000)),
])
def test_feti_equals_monolithic(case, krylov):
    """Theorem 3.1: the FETI solution is the unique solution of the block system; at interface
    tolerance 1e-13 (1e-14 at lambda = 499, where the residual is amplified ~1e3 into the
    pressure fields) the two agree to 1e-10 in lambda and every field."""
    d = Discretization(case)
    mono = solve_monolithic(case, d)
    fe = FETI(case, d).run(krylov=krylov)
    for a, b in zip(mono, fe):
        assert _rel(b["lambda"], a["lambda"]) < 1e-10
        for fa, fb in zip(a["fields"], b["fields"]):
            for xa, xb in zip(fa, fb):
                if xa is not None:
                    assert np.abs(xa - xb).max() < 1e-10 * max(1.0, np.abs(xa).max())


def test_monolithic_solves_the_block_system():
    """Every step's monolithic solution satisfies the block equations of Sec. 2.5 grouped per
    subdomain, K_s x_s + B_s^T lambda = f_s and sum_s B_s x_s = 0, to rounding, on a nearly
    incompressible case (lambda = 499, log-normal permeability) where plain sparse LU alone is
    only good to ~1e-10.  The residual is formed here from the local matrices, not by the solver."""
    case = _lognormal(W.small_case(4, 4, 6, k=2, lame_lambda=499.0, tau=1e-3, n_steps=3,
                                   source="manufactured_t"))
    d = Discretization(case)
    Ls, I = d.locals, d.iface
    Reta = d.initial_Reta()
    for step in solve_monolithic(case, d):
        lam, xs = step["lambda"], step["x"]
        jump = sum(B @ x for B, x in zip(I.Bs, xs))
        assert np.abs(jump).max() <= 1e-14 * max(np.abs(x).max() for x in xs)
        for s, L in enumerate(Ls):
            f = L.rhs(step["t"], Reta[s])
            res = L.K @ xs[s] + I.Bs[s].T @ lam - f
            scale = np.abs(L.K).max() * np.abs(xs[s]).max() + np.abs(f).max()
            assert np.abs(res).max() <= 1e-14 * scale, s
            if L.m.is_poro:
                Reta[s] = L.Reta_of(step["fields"][s][2])


def _small(lame_lambda=49.0, lognormal=False):
    c = W.small_case(4, 4, 2, k=2, lame_lambda=lame_lambda, tau=1e-3, n_steps=1, tol=1e-12)
    if lognormal:
        c = _lognormal(c)
    d = Discretization(c)
    return c, d, FETI(c, d)


@pytest.mark.parametrize("lame_lambda, lognormal", [(49.0, False), (499.0, True)])
def test_operator_properties(lame_lambda, lognormal):
    """F is symmetric with inertia (n_lambda_u, n_lambda_p) on range(P) and the Dirichlet-
    preconditioned operator has a real spectrum >= ~1 there (reading of Algorithm 1 with
    pressure multipliers), also at the large workload's nu = 0.499 with log-normal K."""
    c, d, f = _small(lame_lambda, lognormal)
    I = d.iface
    n = I.n_lambda
    B = np.hstack([Bs.toarray() for Bs in I.Bs])
    assert np.linalg.matrix_rank(B) == n                      # non-redundant multipliers
    for s in I.floating:                                       # K_s R_s = 0
        assert np.abs(d.locals[s].K @ I.Rs[s]).max() < 1e-10
    Fd = f.dense_F()
    assert np.abs(Fd - Fd.T).max() < 1e-10 * np.abs(Fd).max()
    # inertia on range(P): positive for displacement rows, negative for pressure rows
    E = np.eye(n)
    P = np.column_stack([f.P(E[:, j]) for j in range(n)])
    U, sv, _ = np.linalg.svd(P)
    Q = U[:, sv > 0.5]
    ev = np.linalg.eigvalsh(Q.T @ Fd @ Q)
    assert (ev < 0).sum() == I.is_p.sum()
    assert (ev > 0).sum() == Q.shape[1] - I.is_p.sum()
    # preconditioned operator: real spectrum >= ~1 on range(P) (the reason Algorithm 1 is used)
    M = np.column_stack([f.precond(E[:, j]) for j in range(n)])
    mu = np.linalg.eigvals(np.linalg.solve(np.eye(Q.shape[1]), (Q.T @ M @ Q) @ (Q.T @ Fd @ Q)))
    assert mu.real.min() > 0.9 and np.abs(mu.imag).max() < 1e-2 * mu.real.max()


def test_coarse_constraint_and_continuity():
    c, d, f = _small()
    I = d.iface
    Reta = d.initial_Reta()
    fl = [L.rhs(c.tau, Reta[s]) for s, L in enumerate(d.locals)]
    lam, its, hist, dd = f.solve_step(fl, np.zeros(I.n_lambda))
    assert np.abs(I.G.T @ lam - I.e_vector(fl)).max() < 1e-9 * np.abs(I.e_vector(fl)).max()
    xs = f.recover(fl, lam, dd)
    jump = sum(B @ x for B, x in zip(I.Bs, xs))
    assert np.abs(jump).max() < 1e-9 * max(np.abs(x).max() for x in xs)
    for s, L in enumerate(d.locals):  # every local equation K_s x_s + B_s^T lambda = f_s
        res = L.K @ xs[s] + I.Bs[s].T @ lam - fl[s]
        assert np.abs(res).max() < 1e-8 * np.abs(fl[s]).max()


def test_fixed_dofs_do_not_change_solution():
    c, d, f = _small()
    Reta = d.initial_Reta()
    fl = [L.rhs(c.tau, Reta[s]) for s, L in enumerate(d.locals)]
    lam, _, _, dd = f.solve_step(fl, np.zeros(d.iface.n_lambda))
    xs = f.recover(fl, lam, dd)
    f2 = FETI(c, d, fixed_override=lambda s, L: np.array([2 * 4, 2 * 4 + 1, 2 * (L.m.n_unode - 1)]))
    lam2, _, _, dd2 = f2.solve_step(fl, np.zeros(d.iface.n_lambda))
    xs2 = f2.recover(fl, lam2, dd2)
    assert _rel(lam2, lam) < 1e-8
    for a, b in zip(xs, xs2):
        assert np.abs(a - b).max() < 1e-8 * np.abs(a).max()


def test_krylov_against_dense():
    rng = np.random.default_rng(3)
    n = 60
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    A_spd = Q @ np.diag(rng.uniform(1, 50, n)) @ Q.T
    A_ind = Q @ np.diag(np.r_[rng.uniform(1, 50, 40), -rng.uniform(1, 20, 20)]) @ Q.T
    Mi = np.diag(rng.uniform(0.5, 2, n))
    b = rng.normal(size=n)
    x, k, h = pcg(lambda v: A_spd @ v, lambda v: Mi @ v, b, np.zeros(n), 1e-12, np.linalg.norm(b), 500)
    assert _rel(x, np.linalg.solve(A_spd, b)) < 1e-9
    x, k, h = minres(lambda v: A_ind @ v, lambda v: Mi @ v, b, np.zeros(n), 1e-12, np.linalg.norm(b), 500)
    assert _rel(x, np.linalg.solve(A_ind, b)) < 1e-9
    assert abs(h[-1] - np.linalg.norm(b - A_ind @ x)) < 1e-10 * np.linalg.norm(b)


def _three_field_dense(case, L):
    """Dense 3-field local matrix (eta eliminated) in the order [free u, xi, free p], built
    from the full element-level matrices alone (not from the oracle's 4-field system)."""
    A = L.A_full[L.ufree][:, L.ufree].toarray()
    B = L.B_full[:, L.ufree].toarray()
    R = L.R_full.toarray()
    lam, al, c0 = case.lame_lambda, case.alpha, case.c0
    if not L.m.is_poro:
        return np.block([[A, B.T], [B, -R / lam]])
    pf = L.pfree
    Af = L.Af_full.toarray()[np.ix_(pf, pf)]
    Rxp = (al / lam) * R[:, pf]
    Rpp = R[np.ix_(pf, pf)]
    Z = np.zeros((A.shape[0], pf.size))
    return np.block([[A, B.T, Z], [B, -R / lam, Rxp], [Z.T, Rxp.T, -(c0 + al * al / lam) * Rpp - case.tau * Af]])


def test_preconditioner_blocks_against_dense_three_field():
    """The lumped local operator is the interface block of the 3-field matrix, and the
    Dirichlet Schur complement of the oracle's 4-field system equals the 3-field one (eta is
    interior): both against a dense assembly from the element-level matrices."""
    case = W.small_case(3, 4, 2, k=2, lame_lambda=9.0, alpha=0.7, c0=0.4, tau=0.05)
    fe = FETI(case, precond="lumped")
    for s, L in enumerate(fe.Ls):
        bd = fe.bd[s]
        if bd.size == 0:
            continue
        K3 = _three_field_dense(case, L)
        nP = L.m.n_pnode
        b3 = np.where(bd < L.nu, bd, bd - (L.off_p - L.nu - nP)) if L.m.is_poro else bd
        i3 = np.setdiff1d(np.arange(K3.shape[0]), b3)
        Kbb = K3[np.ix_(b3, b3)]
        assert np.abs(fe.Kbb3[s] - Kbb).max() <= 1e-13 * np.abs(Kbb).max(), s
        S3 = Kbb - K3[np.ix_(b3, i3)] @ np.linalg.solve(K3[np.ix_(i3, i3)], K3[np.ix_(i3, b3)])
        S4 = np.stack([fe.S_apply(s, e) for e in np.eye(bd.size)], axis=1)
        assert np.abs(S4 - S3).max() <= 1e-9 * np.abs(S3).max(), s


@pytest.mark.parametrize("precond", ["lumped", "none"])
def test_feti_other_preconditioners_equal_monolithic(precond):
    case = W.small_case(4, 4, 3, k=2, lame_lambda=49.0, tau=1e-3, n_steps=2, tol=1e-12, max_it=3000)
    d = Discretization(case)
    mono = solve_monolithic(case, d)
    fe = FETI(case, d, precond=precond).run()
    for a, b in zip(mono, fe):
        assert _rel(b["lambda"], a["lambda"]) < 1e-8
