"""GPU (CUDA, sm_103a) FP64 path against the CPU oracle, element by element.

Tolerance: 1e-10 relative (max |gpu - oracle| / max |oracle|) for the FP64 path, the bar of
the FP64 arm; PCG runs to tol 1e-13 here so that the iteration error is far below it."""
import numpy as np
import pytest

from paper_2509_06673_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def F():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_06673_gb300 import build
    build.build()
    from paper_2509_06673_gb300 import fetipe
    return fetipe


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def _oracle(case):
    from oracle.monolithic import Discretization
    from oracle.feti import FETI
    d = Discretization(case)
    return d, FETI(case, d)


def _three_field(L, fields, nodes, lam, alpha, c0, tau):
    """3-field block of the oracle's assembly in the library's dof order."""
    n = fields.size
    K = np.zeros((n, n))
    A, B, R, Af = (M.toarray() for M in (L.A_full, L.B_full, L.R_full, L.Af_full))
    idx = np.where(fields <= 1, 2 * nodes + fields, nodes)
    for i in range(n):
        for j in range(n):
            fi, fj, a, b = fields[i], fields[j], idx[i], idx[j]
            if fi <= 1 and fj <= 1:
                K[i, j] = A[a, b]
            elif fi <= 1 and fj == 2:
                K[i, j] = B[b, a]
            elif fi == 2 and fj <= 1:
                K[i, j] = B[a, b]
            elif fi == 2 and fj == 2:
                K[i, j] = -R[a, b] / lam
            elif {fi, fj} == {2, 3}:
                K[i, j] = alpha / lam * R[a, b]
            elif fi == 3 and fj == 3:
                K[i, j] = -(c0 + alpha * alpha / lam) * R[a, b] - tau * Af[a, b]
    return K


@pytest.mark.parametrize("case", [
    W.small_case(2, 2, 2, k=1, lame_lambda=3.0, alpha=0.7, c0=0.4, tau=0.05),
    W.small_case(2, 2, 2, k=2, lame_lambda=49.0, tau=1e-3),
    W.grid_case("perm", 1, 2, 3, 2, order_k=2, perm=[np.linspace(0.5, 2, 12), np.ones(12)]),
])
def test_local_matrices(F, case):
    sol = F.Solver(case)
    sol.assemble()
    d, _ = _oracle(case)
    for s in range(case.nsub):
        f, nd = sol.get_dof_map(s)
        K = sol.get_local_matrix(s)
        ref = _three_field(d.locals[s], f, nd, case.lame_lambda, case.alpha, case.c0, case.tau)
        assert _rel(K, ref) < 1e-13, s
    sol.close()


OPS_CASES = [
    W.config1(),
    W.small_case(4, 4, 3, k=2, lame_lambda=49.0, tau=1e-3),
    W.grid_case("uneven", 3, 4, [2, 4, 3], [3, 2, 4, 3], order_k=1, lame_lambda=5.0, c0=0.5, tau=1e-2),
]


@pytest.mark.parametrize("explicit", [0, 1])
@pytest.mark.parametrize("case", OPS_CASES)
def test_interface_operators(F, case, explicit):
    """explicit = 1: F and the Dirichlet preconditioner applied through the dense local
    operators F_s, S_s built by the multi-right-hand-side band solves."""
    sol = F.Solver(case)
    sol.set_option("explicit", explicit)
    sol.assemble()
    sol.factor()
    d, fe = _oracle(case)
    keys = sol.get_lambda_keys()
    assert np.array_equal(keys, np.array(d.iface.keys, dtype=np.int32))
    rng = np.random.default_rng(0)
    for _ in range(2):
        v = rng.normal(size=d.iface.n_lambda)
        assert _rel(sol.apply_F(v), fe.F(v)) < TOL
        assert _rel(sol.apply_precond(v), fe.precond(v)) < TOL
        assert _rel(sol.apply_projection(v), fe.P(v)) < TOL
    sol.close()


STEP_CASES = [
    W.config1(tol=1e-13),
    W.small_case(4, 4, 3, k=2, lame_lambda=49.0, tau=1e-3, n_steps=3, tol=1e-13),
    W.grid_case("uneven", 3, 4, [2, 4, 3], [3, 2, 4, 3], order_k=1, lame_lambda=5.0, c0=0.5, tau=1e-2,
                n_steps=3, tol=1e-13),
    W.small_case(4, 4, 4, k=2, lame_lambda=9.0, tau=1e-2, n_steps=3, tol=1e-13, source="point",
                 src_node=(6, 5), q_omega=30.0),
]


@pytest.mark.parametrize("explicit", [0, 1])
@pytest.mark.parametrize("case", STEP_CASES)
def test_steps_match_oracle(F, case, explicit):
    from oracle.monolithic import solve_monolithic
    d, _ = _oracle(case)
    mono = solve_monolithic(case, d)
    sol = F.Solver(case)
    sol.set_option("explicit", explicit)
    sol.assemble()
    sol.factor()
    for n in range(case.n_steps):
        st = sol.step()
        assert st["true_rel_residual"] < 1e-11
        lam = sol.get_lambda()
        assert _rel(lam, mono[n]["lambda"]) < TOL, n
        fields = F.split_fields(case, *sol.get_fields())
        for s, (gu, gxi, geta, gp) in enumerate(fields):
            u, xi, eta, p = mono[n]["fields"][s]
            scale = max(np.abs(u).max(), 1e-300)
            assert np.abs(gu - u).max() < TOL * scale, (n, s)
            assert np.abs(gxi - xi).max() < TOL * max(np.abs(xi).max(), 1.0), (n, s)
            if eta is not None:
                assert np.abs(gp - p).max() < TOL * max(np.abs(p).max(), 1e-300), (n, s)
                assert np.abs(geta - eta).max() < TOL * max(np.abs(eta).max(), 1e-300), (n, s)
    sol.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_blocked_and_rowstep_solves_agree(F, precision):
    """The blocked sweeps (inverse diagonal blocks) and the row-step sweeps solve the same
    band systems: F applied both ways agrees to rounding, on subdomains with partial last
    blocks and several band widths (uneven meshes)."""
    case = W.grid_case("uneven", 3, 4, [5, 7, 6], [6, 5, 7, 6], order_k=2, lame_lambda=49.0, tau=1e-3,
                       precision=precision)
    sol = F.Solver(case)
    sol.assemble()
    sol.factor()
    v = np.random.default_rng(3).normal(size=sol.sizes.n_lambda)
    sol.set_option("ir_sweeps", 0)
    a = sol.apply_F(v)
    sol.set_option("solve_kernel", 0)
    b = sol.apply_F(v)
    tol = 1e-12 if precision == "fp64" else 1e-5
    assert _rel(a, b) < tol
    sol.close()
