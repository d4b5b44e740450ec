"""Per-subdomain output and checkpoint / restore of the time-stepping state."""
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


def test_get_subdomain_matches_split_fields(F):
    case = W.grid_case("uneven", 3, 4, [3, 5, 4], [4, 3, 5, 4], order_k=2, lame_lambda=9.0, tau=1e-2,
                       n_steps=2, source="manufactured_t")
    sol = F.Solver(case)
    sol.assemble()
    sol.factor()
    sol.step()
    parts = F.split_fields(case, *sol.get_fields())
    for s in range(case.nsub):
        for a, b in zip(sol.get_subdomain(s), parts[s]):
            assert np.array_equal(a, b)
    with pytest.raises(F.FetipeError):
        sol.get_subdomain(case.nsub)
    sol.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_checkpoint_restore_continues_bit_for_bit(F, tmp_path, precision):
    """Run 5 steps; separately run 3, checkpoint, restore into a fresh handle and run 2: the
    same lambda and fields bit for bit (the learned guess in use, so the network state and
    the source history travel too)."""
    case = W.small_case(4, 4, 4, k=2, lame_lambda=9.0, tau=2e-3, n_steps=5, tol=1e-10, source="point",
                        q_omega=25.0, precision=precision)
    case = case.with_(src_node=W.point_source_node(case, 1000))

    def fresh():
        sol = F.Solver(case)
        sol.assemble()
        sol.factor()
        sol.mlp_init(7)
        sol.learned_use(True)
        return sol

    ref = fresh()
    for _ in range(5):
        ref.step()
    lam_ref, fields_ref = ref.get_lambda(), ref.get_fields()
    ref.close()

    a = fresh()
    for _ in range(3):
        a.step()
    path = tmp_path / "state.ckpt"
    a.checkpoint(path)
    a.close()
    b = fresh()
    b.restore(path)
    sts = [b.step() for _ in range(2)]
    assert sts[-1]["step"] == 5
    assert np.array_equal(b.get_lambda(), lam_ref)
    for x, y in zip(b.get_fields(), fields_ref):
        assert np.array_equal(x, y)
    b.close()


def test_restore_rejects_other_problem(F, tmp_path):
    c1 = W.small_case(2, 2, 3, k=2, n_steps=1)
    c2 = W.small_case(2, 2, 4, k=2, n_steps=1)
    s1 = F.Solver(c1)
    s1.assemble()
    s1.factor()
    s1.step()
    s1.checkpoint(tmp_path / "c1")
    s1.close()
    s2 = F.Solver(c2)
    with pytest.raises(F.FetipeError):
        s2.restore(tmp_path / "c1")          # before fp_assemble: state error
    s2.assemble()
    with pytest.raises(F.FetipeError):
        s2.restore(tmp_path / "c1")          # other sizes
    (tmp_path / "bad").write_bytes(b"not a checkpoint")
    with pytest.raises(F.FetipeError):
        s2.restore(tmp_path / "bad")
    s2.close()
    # same problem: a truncated file and one with bytes appended are rejected, the file
    # itself is accepted
    good = (tmp_path / "c1").read_bytes()
    (tmp_path / "short").write_bytes(good[:-1])
    (tmp_path / "long").write_bytes(good + b"\0")
    s3 = F.Solver(c1)
    s3.assemble()
    for name in ("short", "long"):
        with pytest.raises(F.FetipeError) as e:
            s3.restore(tmp_path / name)
        assert e.value.status == F.FP_ERR_INVALID, name
    s3.restore(tmp_path / "c1")
    s3.close()


def test_set_initial_matches_oracle(F):
    """Given initial fields (smooth, defined from global coordinates so that shared nodes
    agree): the GPU steps from R eta^0 = (c0 p0 + alpha div u0, phi_i) match the oracle's
    monolithic solve from the same fields (FP64, 1e-10)."""
    from oracle.monolithic import Discretization, solve_monolithic
    case = W.grid_case("init", 2, 2, [3, 4], [2, 3], order_k=2, lame_lambda=7.0, alpha=0.8, c0=0.3,
                       tau=1e-2, n_steps=2, tol=1e-13)
    d = Discretization(case)
    initial, u_all, p_all = [], [], []
    for L in d.locals:
        m = L.m
        ux, uy = m.unode_xy()
        px, py = m.pnode_xy()
        u0 = np.stack([np.sin(3 * ux) * np.cos(2 * uy), ux * uy], axis=1)
        p0 = np.cos(px + py) if m.is_poro else None
        initial.append((u0, p0))
        u_all.append(u0.ravel())
        p_all.append(p0 if m.is_poro else np.zeros(m.n_pnode))
    mono = solve_monolithic(case, d, initial=initial)
    ref0 = solve_monolithic(case, d)
    sol = F.Solver(case)
    sol.assemble()
    sol.factor()
    sol.set_initial(np.concatenate(u_all), np.concatenate(p_all))
    got_u = sol.get_fields()[0]
    assert np.array_equal(got_u, np.concatenate(u_all))
    for n in range(case.n_steps):
        sol.step()
        lam = sol.get_lambda()
        scale = np.abs(mono[n]["lambda"]).max()
        assert np.abs(lam - mono[n]["lambda"]).max() < 1e-10 * scale, n
        fields = F.split_fields(case, *sol.get_fields())
        for s, (gu, gxi, geta, gp) in enumerate(fields):
            u, xi, eta, p = mono[n]["fields"][s]
            assert np.abs(gu - u).max() < 1e-10 * np.abs(u).max(), (n, s)
            if eta is not None:
                assert np.abs(gp - p).max() < 1e-10 * np.abs(p).max(), (n, s)
                assert np.abs(geta - eta).max() < 1e-10 * np.abs(eta).max(), (n, s)
    # the initial data matters: the default initial state gives another first step
    assert np.abs(mono[0]["lambda"] - ref0[0]["lambda"]).max() > 1e-6 * np.abs(ref0[0]["lambda"]).max()
    sol.close()


def test_step_moves_only_scalars_across_the_host_link(F):
    """fp_step reports its own host<->device copies: the per-step scalars and loop flags in,
    flags, scalars and the status word out -- bytes, not vectors -- on the graph and the
    stream path."""
    case = W.small_case(3, 4, 4, k=2, n_steps=2)
    for graph in (1, 0):
        sol = F.Solver(case)
        sol.set_option("graph", graph)
        sol.assemble()
        sol.factor()
        for _ in range(2):
            st = sol.step()
            assert 0 < st["h2d_bytes"] <= 1024, (graph, st)
            assert 0 < st["d2h_bytes"] <= 64 * 1024, (graph, st)
            assert st["h2d_bytes"] < 8 * sol.sizes.n_lambda
        sol.close()
