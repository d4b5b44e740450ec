"""Lumped preconditioner (Sec. 3.3: W B K_bb B^T W, no local solve) against the oracle, and the
autotuned preconditioner choice (probe runs of Algorithm 1 with each candidate)."""
import numpy as np
import pytest

from paper_2509_06673_gb300 import workloads as W

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("case", [
    W.small_case(4, 4, 3, k=2, lame_lambda=49.0, tau=1e-3, precond="lumped"),
    W.grid_case("uneven", 3, 4, [2, 4, 3], [3, 2, 4, 3], order_k=1, lame_lambda=5.0, c0=0.5, tau=1e-2,
                precond="lumped"),
])
def test_lumped_apply_matches_oracle(F, case):
    from oracle.feti import FETI
    fe = FETI(case, precond="lumped")
    sol = F.Solver(case)
    sol.assemble()
    sol.factor()
    rng = np.random.default_rng(2)
    for _ in range(2):
        v = rng.normal(size=sol.sizes.n_lambda)
        assert _rel(sol.apply_precond(v), fe.precond(v)) < 1e-10
    sol.close()


@pytest.mark.parametrize("precision,explicit,tolerance", [("fp64", 0, 1e-10), ("fp64", 1, 1e-10),
                                                          ("mixed", 1, 1e-8)])
def test_lumped_steps_match_oracle(F, precision, explicit, tolerance):
    from oracle.monolithic import Discretization, solve_monolithic
    case = W.small_case(4, 4, 4, k=2, lame_lambda=49.0, tau=1e-3, n_steps=2, tol=1e-13, precond="lumped",
                        source="manufactured_t", precision=precision, max_it=4000)
    d = Discretization(case)
    mono = solve_monolithic(case, d)
    sol = F.Solver(case)
    sol.set_option("explicit", explicit)
    sol.set_option("ir_eps", 1e-15)
    sol.assemble()
    sol.factor()
    assert sol.tuning()["precond"] == F.FP_PRECOND_LUMPED
    for n in range(case.n_steps):
        st = sol.step()
        assert st["true_rel_residual"] <= case.tol
        assert _rel(sol.get_lambda(), mono[n]["lambda"]) < tolerance, n
    sol.close()


def test_auto_preconditioner(F):
    from oracle.monolithic import Discretization, solve_monolithic
    case = W.small_case(4, 4, 4, k=2, lame_lambda=49.0, tau=1e-3, n_steps=2, tol=1e-13, precond="auto",
                        source="manufactured_t", max_it=4000)
    sol = F.Solver(case)
    sol.assemble()
    sol.factor()
    tun = sol.tuning()
    assert tun["precond"] in (F.FP_PRECOND_DIRICHLET, F.FP_PRECOND_LUMPED)
    assert all(0.0 < r < 1.0 for r in tun["precond_rate"])
    assert all(m > 0.0 for m in tun["precond_ms_per_it"])
    # the Dirichlet preconditioner contracts faster per iteration than the lumped one
    assert tun["precond_rate"][0] < tun["precond_rate"][1]
    mono = solve_monolithic(case, Discretization(case))
    for n in range(case.n_steps):
        sol.step()
        assert _rel(sol.get_lambda(), mono[n]["lambda"]) < 1e-10, n
    sol.close()


@pytest.mark.parametrize("tile", [16, 32])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_explicit_build_tile_widths(F, tile, precision):
    """Both tile widths of the explicit-operator build give the band-solve operators
    (F and the Dirichlet preconditioner) on uneven subdomains with partial tiles."""
    case = W.grid_case("uneven", 3, 4, [5, 7, 6], [6, 5, 7, 6], order_k=2, lame_lambda=49.0, tau=1e-3,
                       precision=precision)
    ref = F.Solver(case)
    ref.assemble()
    ref.factor()
    sol = F.Solver(case)
    sol.set_option("explicit", 1)
    sol.set_option("explicit_tile", tile)
    sol.assemble()
    sol.factor()
    v = np.random.default_rng(4).normal(size=sol.sizes.n_lambda)
    tol = 1e-12 if precision == "fp64" else 1e-9
    # accurate F: FP64 operators in both precisions
    assert _rel(sol.apply_F(v), ref.apply_F(v)) < tol
    # the preconditioner: FP64 S_s (fp64), BF16 symmetric tiles (mixed default) against FP32 band
    # solves: within BF16's rounding (2^-9)
    assert _rel(sol.apply_precond(v), ref.apply_precond(v)) < (1e-12 if precision == "fp64" else 1e-2)
    sol.close()
    if precision == "mixed":
        # FP32 tiles (precond_bf16 0): within FP32 rounding of the band solves
        sol = F.Solver(case)
        sol.set_option("explicit", 1)
        sol.set_option("explicit_tile", tile)
        sol.set_option("precond_bf16", 0)
        sol.assemble()
        sol.factor()
        assert _rel(sol.apply_precond(v), ref.apply_precond(v)) < 1e-5
        sol.close()
    ref.close()
