"""Autotuner: the launch shapes it picks are legal, user-pinned shapes are kept, and the
results do not depend on the shape (every subdomain's solve runs the same arithmetic in the
same order whatever the warps per CTA, stage size or CTAs per SM), so they agree bit for bit."""
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


def _solve(F, case, precision, opts):
    sol = F.Solver(case, precision=precision)
    for k, v in opts:
        sol.set_option(k, v)
    sol.assemble()
    sol.factor()
    tun = sol.tuning()
    its = [sol.step()["iterations"] for _ in range(2)]
    lam = sol.get_lambda()
    u = sol.get_fields()[0]
    sol.close()
    return tun, its, lam, u


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_autotuned_shape_is_legal_and_exact(F, precision):
    case = W.small_case(4, 4, 6, k=2, lame_lambda=49.0, tau=1e-3, n_steps=2, tol=1e-10,
                        source="manufactured_t")
    tun, its, lam, u = _solve(F, case, precision, ())
    assert tun["candidates"] >= 2 and tun["solve_ms"] > 0 and tun["factor_ms"] > 0
    assert tun["solve_wpc"] in (1, 2, 4, 8) and tun["solve_ctas_per_sm"] in (1, 2)
    esz = 4 if precision == "mixed" else 8
    assert tun["solve_chunk"] % 1024 == 0 and tun["solve_chunk"] >= 1024 * esz
    assert tun["solve_wpc"] * 3 * (tun["solve_chunk"] + 8) * tun["solve_ctas_per_sm"] <= 220 * 1024
    assert tun["factor_nb"] in (8, 16, 32, 64)
    # pinned shapes, no tuning: the same numbers bit for bit
    for opts in ((("autotune", 0), ("factor_nb", tun["factor_nb"])),
                 (("autotune", 0), ("solve_wpc", 1), ("solve_chunk", 16384), ("factor_nb", tun["factor_nb"])),
                 (("solve_wpc", 2), ("solve_cps", 2), ("factor_nb", tun["factor_nb"]))):
        t2, its2, lam2, u2 = _solve(F, case, precision, opts)
        assert its2 == its
        assert np.array_equal(lam2, lam) and np.array_equal(u2, u)
        for k, v in opts:
            if k == "solve_wpc":
                assert t2["solve_wpc"] == v


def test_factor_width_does_not_change_the_factor_beyond_rounding(F):
    """Different panel widths reorder the trailing-update sums: the solutions agree to
    rounding (FP64 path, 1e-12 relative)."""
    case = W.small_case(4, 4, 6, k=2, lame_lambda=49.0, tau=1e-3, n_steps=2, tol=1e-12,
                        source="manufactured_t")
    _, _, lam8, _ = _solve(F, case, "fp64", (("factor_nb", 8),))
    _, _, lam32, _ = _solve(F, case, "fp64", (("factor_nb", 32),))
    assert np.abs(lam8 - lam32).max() <= 1e-10 * np.abs(lam32).max()
