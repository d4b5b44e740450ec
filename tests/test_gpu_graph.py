"""CUDA graph per time step: the captured step (prologue, Algorithm 1 and its restarts as
nested conditional WHILE nodes, recovery) against the same kernels driven from the host.
Both run identical launches in identical order with fixed-order reductions, so results
must agree bit for bit, and the device-side loops must stop at the same bounds."""
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


def _run(F, case, graph, n, opts=(), precision=None, allow_failure=False, theta=None):
    sol = F.Solver(case, precision=precision)
    sol.set_option("graph", graph)
    for k, v in opts:
        sol.set_option(k, v)
    sol.assemble()
    sol.factor()
    if theta is not None:
        sol.mlp_set_params(theta)
        sol.learned_use(True)
    stats, restarts = [], []
    for _ in range(n):
        stats.append(sol.step(allow_failure=allow_failure))
        restarts.append(int(sol.step_timing()[3]))
    lam = sol.get_lambda()
    fields = sol.get_fields()
    sol.close()
    return stats, restarts, lam, fields


def _same(a, b):
    sa, ra, la, fa = a
    sb, rb, lb, fb = b
    assert [s["iterations"] for s in sa] == [s["iterations"] for s in sb]
    assert [s["stagnations"] for s in sa] == [s["stagnations"] for s in sb]
    assert [s["status"] for s in sa] == [s["status"] for s in sb]
    assert ra == rb
    assert np.array_equal(la, lb)
    for x, y in zip(fa, fb):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("explicit", [0, 1])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_matches_stream_bitwise(F, precision, explicit):
    case = W.small_case(3, 4, 5, k=2, lame_lambda=49.0, tau=1e-3, n_steps=4, tol=1e-10,
                        source="manufactured_t")
    opts = (("explicit", explicit),)
    a = _run(F, case, 0, 4, opts=opts, precision=precision)
    b = _run(F, case, 1, 4, opts=opts, precision=precision)
    _same(a, b)
    assert all(s["true_rel_residual"] <= 1e-10 for s in b[0])


def test_graph_restarts_match_stream(F):
    """Mixed precision with an FP32-factored operator inside the loop and a tight tolerance:
    the recursive residual runs ahead of the true one, so steps restart; graph and stream
    take the same restarts."""
    case = W.small_case(3, 4, 5, k=2, lame_lambda=499.0, tau=1e-3, n_steps=3, tol=1e-13,
                        source="manufactured_t")
    opts = (("factor_fp64", 0), ("ir_eps", 1e-15))
    a = _run(F, case, 0, 3, opts=opts, precision="mixed", allow_failure=True)
    b = _run(F, case, 1, 3, opts=opts, precision="mixed", allow_failure=True)
    _same(a, b)


def test_graph_stagnation_stops_match_stream(F):
    """A tiny stagnation window makes rounds stop early and restart from the true residual;
    the step still converges and graph and stream agree."""
    case = W.small_case(3, 4, 5, k=2, lame_lambda=49.0, tau=1e-3, n_steps=3, tol=1e-10,
                        source="manufactured_t")
    opts = (("stag_window", 3), ("max_restarts", 64))
    a = _run(F, case, 0, 3, opts=opts, precision="mixed", allow_failure=True)
    b = _run(F, case, 1, 3, opts=opts, precision="mixed", allow_failure=True)
    _same(a, b)
    assert sum(s["stagnations"] for s in b[0]) >= 1
    assert all(s["restarts"] >= s["stagnations"] for s in b[0])


def test_graph_loop_bounds(F):
    """An unreachable tolerance: the device loops stop at max_it and at max_restarts, the
    step reports not-converged, and graph and stream agree."""
    case = W.small_case(3, 4, 4, k=2, lame_lambda=9.0, tau=1e-2, n_steps=2, tol=1e-30, max_it=37,
                        source="manufactured_t")
    opts = (("pcg_chunk", 5), ("max_restarts", 2))
    for precision in ("fp64", "mixed"):
        a = _run(F, case, 0, 2, opts=opts, precision=precision, allow_failure=True)
        b = _run(F, case, 1, 2, opts=opts, precision=precision, allow_failure=True)
        _same(a, b)
        for s, r in zip(b[0], b[1]):
            assert s["status"] == F.FP_ERR_NOT_CONVERGED
            assert s["iterations"] <= 37 + 5
            assert r <= 2


def test_graph_learned_matches_stream(F):
    """The learned-guess variant of the step graph (features, MLP, guess selection inside the graph)."""
    case = W.small_case(4, 4, 4, k=2, lame_lambda=9.0, tau=2e-3, n_steps=12, tol=1e-8, source="point",
                        q_omega=25.0)
    case = case.with_(src_node=W.point_source_node(case, 1000))
    rec = F.Solver(case)
    rec.assemble()
    rec.factor()
    rec.learned_record(True, max_samples=200_000)
    for _ in range(8):
        rec.step()
    rec.learned_train(epochs=3, batch=512, lr=2e-3, seed=1)
    theta = rec.mlp_get_params()
    rec.close()
    a = _run(F, case, 0, 6, theta=theta)
    b = _run(F, case, 1, 6, theta=theta)
    _same(a, b)
    assert [s["lambda0_learned"] for s in a[0]] == [s["lambda0_learned"] for s in b[0]]


def test_graph_profiling_counts_prologue_solves(F):
    case = W.small_case(3, 4, 5, k=2, lame_lambda=9.0, tau=1e-2, n_steps=3, tol=1e-10)
    sol = F.Solver(case, precision="mixed")
    sol.assemble()
    sol.factor()
    sol.set_profiling(True)
    for _ in range(3):
        sol.step()
    st = sol.kernel_stats(0)
    sol.close()
    assert st["launches"] >= 3 and st["total_ms"] > 0


def test_graph_kernel_launch_count(F):
    """fp_step reports the kernels the step launched: the step graph's kernel nodes, the outer
    loop body's per round and the inner body's per execution (counted on the device).  With
    pcg_chunk = 1 every inner body is one iteration of Algorithm 1, so two steps that differ in
    iterations but not in restarts differ in launches by a whole number of bodies, and each body
    holds at least the 14 kernels of one iteration (explicit operators, mixed precision: F 2,
    projection with its dot product 4, update with the preconditioner's W scaling 1,
    preconditioner 2, projection 4, p update 1);
    without the graph nothing is counted."""
    case = W.small_case(4, 4, 3, k=2, lame_lambda=49.0, tau=1e-3, n_steps=3, tol=1e-10, precision="mixed",
                        source="manufactured_t")
    sol = F.Solver(case)
    sol.set_option("pcg_chunk", 1)
    sol.set_option("explicit", 1)
    sol.assemble()
    sol.factor()
    sts = [sol.step() for _ in range(3)]
    for st in sts:
        assert st["kernel_launches"] >= 14 * st["iterations"]
    same = [st for st in sts if st["restarts"] == sts[0]["restarts"]]
    if len(same) >= 2 and same[0]["iterations"] != same[1]["iterations"]:
        diff = same[0]["kernel_launches"] - same[1]["kernel_launches"]
        per_body = diff / (same[0]["iterations"] - same[1]["iterations"])
        assert per_body == int(per_body) and per_body >= 14
    sol.set_option("graph", 0)
    assert sol.step()["kernel_launches"] == -1
    sol.close()
