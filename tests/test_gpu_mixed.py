"""Mixed-precision path (FP32 local factors and solves, FP64 outer PCG, coarse problem and
refinement residuals) against the FP64 oracle.  Bar: 1e-8 relative in lambda, u, xi, eta,
p, the accuracy target of the mixed arm; the true FP64 interface residual must meet tol.
The interface tolerance is 1e-13 as in the FP64 tests: the condition number of the
preconditioned interface operator (up to ~1e3 at lambda = 499) amplifies the residual
into the field errors."""
import numpy as np
import pytest

from paper_2509_06673_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-8


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


CASES = [
    W.small_case(4, 4, 4, k=2, lame_lambda=49.0, tau=1e-3, n_steps=3, tol=1e-13, precision="mixed",
                 source="manufactured_t"),
    W.small_case(4, 4, 6, k=2, lame_lambda=499.0, tau=1e-3, n_steps=2, tol=1e-13, precision="mixed",
                 source="manufactured_t", perm=None).with_(
        perm=[np.exp(np.sin(np.arange(72) * (s + 1))) for s in range(16)]),
    W.grid_case("uneven mixed", 3, 4, [3, 5, 4], [4, 3, 5, 4], order_k=2, lame_lambda=9.0, tau=1e-2,
                n_steps=2, tol=1e-13, precision="mixed", source="manufactured_t"),
]


@pytest.mark.parametrize("explicit", [0, 1])
@pytest.mark.parametrize("case", CASES)
def test_mixed_steps_match_oracle(F, case, explicit):
    """explicit = 1: the PCG loop applies F and the preconditioner through FP32 dense local
    operators; the accurate applies keep the refined band solves."""
    from oracle.monolithic import Discretization, solve_monolithic
    d = Discretization(case)
    mono = solve_monolithic(case, d)
    sol = F.Solver(case)
    sol.set_option("ir_eps", 1e-15)
    sol.set_option("explicit", explicit)
    sol.assemble()
    sol.factor()
    for n in range(case.n_steps):
        st = sol.step()
        assert st["true_rel_residual"] <= case.tol
        assert _rel(sol.get_lambda(), mono[n]["lambda"]) < TOL, n
        fields = F.split_fields(case, *sol.get_fields())
        for s, (gu, gxi, geta, gp) in enumerate(fields):
            u, xi, eta, p = mono[n]["fields"][s]
            assert np.abs(gu - u).max() < TOL * np.abs(u).max(), (n, s)
            assert np.abs(gxi - xi).max() < TOL * max(np.abs(xi).max(), 1.0), (n, s)
            if eta is not None:
                assert np.abs(gp - p).max() < TOL * max(np.abs(p).max(), 1e-300), (n, s)
                assert np.abs(geta - eta).max() < TOL * max(np.abs(eta).max(), 1e-300), (n, s)
    sol.close()


def test_mixed_operator_accuracy(F):
    """The refined F apply of the mixed path matches the oracle's FP64 F."""
    from oracle.monolithic import Discretization
    from oracle.feti import FETI
    case = CASES[1]
    sol = F.Solver(case)
    sol.assemble()
    sol.factor()
    fe = FETI(case, Discretization(case))
    v = np.random.default_rng(1).normal(size=sol.sizes.n_lambda)
    assert _rel(sol.apply_F(v), fe.F(v)) < 1e-9
    sol.set_option("ir_sweeps", 0)
    e0 = _rel(sol.apply_F(v), fe.F(v))
    assert 1e-12 < e0 < 1e-2   # plain FP32 solves: visibly less accurate, still close
    sol.close()


@pytest.mark.parametrize("nsub, cells", [(8, 3), (16, 2)])
def test_two_float_coarse_projection(F, nsub, cells):
    """Mixed precision multiplies by (G^T G)^{-1} from hi/lo FP32 upper tiles with error-free
    products and sums: P v agrees with the oracle's FP64 projector (and with the library's FP64
    dense product, option coarse_2f = 0) to 1e-12, with 36 and 196 floating subdomains
    (coarse orders 108 and 588: several 32 x 32 tile rows and a ragged last one)."""
    from oracle.monolithic import Discretization
    from oracle.feti import FETI
    case = W.small_case(nsub, nsub, cells, k=1, lame_lambda=49.0, tau=1e-3, precision="mixed")
    sol = F.Solver(case)
    sol.assemble()
    sol.factor()
    assert sol.sizes.n_floating == (nsub - 2) ** 2
    fe = FETI(case, Discretization(case))
    rng = np.random.default_rng(11)
    for _ in range(3):
        v = rng.normal(size=sol.sizes.n_lambda)
        got = sol.apply_projection(v)
        assert _rel(got, fe.P(v)) < 1e-12
        sol.set_option("coarse_2f", 0)
        ref = sol.apply_projection(v)
        sol.set_option("coarse_2f", 1)
        assert _rel(got, ref) < 1e-12
        # the projector's defining property: G^T P v = 0 (P v orthogonal to range(G))
        G = fe.I.G
        assert np.abs(G.T @ got).max() < 1e-11 * np.abs(G.T @ v).max()
    sol.close()


# half bandwidths 75 (one 128-row tile) and 175 (two, as on the large workload's 24 x 24 cells)
TC_CASES = [CASES[1], W.small_case(3, 4, 16, k=2, lame_lambda=49.0, tau=1e-3, precision="mixed",
                                   source="manufactured_t")]


@pytest.mark.parametrize("case", TC_CASES)
def test_tensor_core_factorisation(F, case):
    """FP32 band factors with the trailing updates on the tensor cores (tcgen05 TF32 tiles, 3xTF32
    split) against the CUDA-core FP32 factorisation and the oracle: the unrefined local solves of
    both are equally close to the FP64 F and Dirichlet preconditioner, and the refined F apply
    meets the FP64 bar."""
    from oracle.monolithic import Discretization
    from oracle.feti import FETI
    fe = FETI(case, Discretization(case))
    v = np.random.default_rng(5).normal(size=fe.I.n_lambda)
    errs = {}
    for tc in (1, 0):
        sol = F.Solver(case)
        sol.set_option("factor_fp64", 0)
        sol.set_option("factor_tc", tc)
        sol.assemble()
        sol.factor()
        ms = sol.tuning()["factor_tc_ms"]
        assert (ms[0] > 0 and ms[1] > 0) == bool(tc)
        assert _rel(sol.apply_F(v), fe.F(v)) < 1e-9
        sol.set_option("ir_sweeps", 0)
        errs[tc] = (_rel(sol.apply_F(v), fe.F(v)), _rel(sol.apply_precond(v), fe.precond(v)))
        sol.close()
    for k in range(2):
        assert errs[1][k] < 1e-2 and errs[1][k] < 20 * errs[0][k] + 1e-12, errs


def test_tensor_core_factorisation_steps(F):
    """Both FP32 factors on the tensor cores (factor_fp64 = 0): steps match the oracle at 1e-8."""
    from oracle.monolithic import Discretization, solve_monolithic
    case = CASES[0]
    mono = solve_monolithic(case, Discretization(case))
    sol = F.Solver(case)
    sol.set_option("factor_fp64", 0)
    sol.set_option("ir_eps", 1e-15)
    sol.assemble()
    sol.factor()
    assert min(sol.tuning()["factor_tc_ms"]) > 0
    for n in range(case.n_steps):
        st = sol.step()
        assert st["true_rel_residual"] <= case.tol
        assert _rel(sol.get_lambda(), mono[n]["lambda"]) < TOL, n
        for s, (gu, gxi, geta, gp) in enumerate(F.split_fields(case, *sol.get_fields())):
            u, xi, eta, p = mono[n]["fields"][s]
            assert np.abs(gu - u).max() < TOL * np.abs(u).max(), (n, s)
            if eta is not None:
                assert np.abs(gp - p).max() < TOL * max(np.abs(p).max(), 1e-300), (n, s)
    sol.close()


def test_two_float_explicit_accurate_apply(F):
    """With explicit operators, the accurate F applies of mixed precision multiply by F_s kept
    as hi/lo FP32 symmetric tiles (two-float arithmetic): F v agrees with the oracle's FP64 F
    and with the FP64 F_s product (explicit_2f = 0) to 1e-12."""
    from oracle.monolithic import Discretization
    from oracle.feti import FETI
    case = CASES[1]
    sol = F.Solver(case)
    sol.set_option("explicit", 1)
    sol.assemble()
    sol.factor()
    fe = FETI(case, Discretization(case))
    rng = np.random.default_rng(4)
    for _ in range(2):
        v = rng.normal(size=sol.sizes.n_lambda)
        got = sol.apply_F(v)
        assert _rel(got, fe.F(v)) < 1e-12
        sol.set_option("explicit_2f", 0)
        ref = sol.apply_F(v)
        sol.set_option("explicit_2f", 1)
        assert _rel(got, ref) < 1e-12
    sol.close()


def test_bf16_preconditioner_steps(F):
    """The Dirichlet preconditioner's S_s tiles in BF16 (option precond_bf16): the preconditioner
    only steers Algorithm 1, so the steps still match the oracle at 1e-8, and the iteration count
    stays within a few of the FP32 tiles'."""
    from oracle.monolithic import Discretization, solve_monolithic
    case = CASES[1]
    mono = solve_monolithic(case, Discretization(case))
    its = {}
    for bf in (0, 1):
        sol = F.Solver(case)
        sol.set_option("explicit", 1)
        sol.set_option("precond_bf16", bf)
        sol.set_option("ir_eps", 1e-15)
        sol.assemble()
        sol.factor()
        its[bf] = []
        for n in range(case.n_steps):
            st = sol.step()
            its[bf].append(st["iterations"])
            assert st["true_rel_residual"] <= case.tol
            assert _rel(sol.get_lambda(), mono[n]["lambda"]) < TOL, (bf, n)
            for s, (gu, gxi, geta, gp) in enumerate(F.split_fields(case, *sol.get_fields())):
                u, xi, eta, p = mono[n]["fields"][s]
                assert np.abs(gu - u).max() < TOL * np.abs(u).max(), (bf, n, s)
                if eta is not None:
                    assert np.abs(gp - p).max() < TOL * max(np.abs(p).max(), 1e-300), (bf, n, s)
        sol.close()
    assert sum(its[1]) <= 1.25 * sum(its[0]) + 4, its


def test_two_float_build_of_F(F):
    """The FP64 F_s behind the accurate applies built in two-float arithmetic from the FP64
    factor split into hi/lo FP32 pairs (explicit_df = 1, the default) against the same build in
    FP64 arithmetic (explicit_df = 0) and the oracle's F, at lambda = 499 (log-normal
    permeability): the accurate F applies agree to 1e-12, and the mixed steps still match the
    oracle's monolithic solution at 1e-8."""
    from oracle.monolithic import Discretization, solve_monolithic
    from oracle.feti import FETI
    case = CASES[1]
    disc = Discretization(case)
    fe = FETI(case, disc)
    out = {}
    for df in (1, 0):
        sol = F.Solver(case)
        sol.set_option("explicit", 1)
        sol.set_option("explicit_df", df)
        sol.set_option("ir_eps", 1e-15)
        sol.assemble()
        sol.factor()
        assert sol.tuning()["mrhs_prec"][0] == (2 if df else 0)
        v = np.random.default_rng(7).normal(size=sol.sizes.n_lambda)
        out[df] = sol.apply_F(v)
        assert _rel(out[df], fe.F(v)) < 1e-12, df
        if df:
            mono = solve_monolithic(case, disc)
            for n in range(case.n_steps):
                st = sol.step()
                assert st["true_rel_residual"] <= case.tol
                assert _rel(sol.get_lambda(), mono[n]["lambda"]) < TOL, n
        sol.close()
    assert _rel(out[1], out[0]) < 1e-12
