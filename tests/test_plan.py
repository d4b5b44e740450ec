"""fp_plan: the library's host topology (dof numbering, multiplier rows of the jump operator B,
floating subdomains) computed without a CUDA device, checked bit for bit against the oracle's
Interface on small cases, against closed-form counts on the 64 x 64-subdomain workload and
against a brute-force node-multiplicity count on the uneven 32 x 32 workload."""
import numpy as np
import pytest

from paper_2509_06673_gb300 import fetipe as F
from paper_2509_06673_gb300 import workloads as W


SMALL = [
    W.config1(n_steps=1),
    W.small_case(2, 2, 4, k=1),
    W.small_case(3, 4, 5, k=2),                                   # floating subdomains, cross points
    W.small_case(3, 4, 3, k=2).with_(poro_rows=1),                # one poroelastic row
    W.small_case(3, 6, 3, k=1).with_(poro_rows=4),
    W.grid_case("uneven 4x4", 4, 4, [2, 5, 3, 4], [3, 2, 4, 3], order_k=2),
    W.grid_case("uneven 5x4", 5, 4, [4, 2, 3, 2, 5], [2, 6, 3, 2], order_k=1).with_(poro_rows=3),
]


@pytest.mark.parametrize("case", SMALL, ids=lambda c: c.name)
def test_plan_matches_oracle_interface(case):
    from oracle.monolithic import Discretization
    s, keys = F.plan(case, keys=True)
    d = Discretization(case)
    assert np.array_equal(keys, np.array(d.iface.keys, dtype=np.int32).reshape(-1, 6))
    assert s.n_lambda == d.iface.n_lambda
    assert s.n_lambda_p == int(d.iface.is_p.sum())
    assert s.n_floating == len(d.iface.floating)
    assert s.nsub == len(d.meshes)
    assert s.n_unode_total == sum(m.n_unode for m in d.meshes)
    assert s.n_pnode_total == sum(m.n_pnode for m in d.meshes)
    # 3-field (u, xi, p) dofs = the oracle's 4-field dofs without eta (one per P1 node)
    assert s.n_dofs == sum(L.n - (m.n_pnode if m.is_poro else 0) for L, m in zip(d.locals, d.meshes))


def _brute_force_counts(case):
    """Multiplier and floating counts from node multiplicities on the global grids: a node
    shared by m subdomains carries m - 1 rows (per displacement component), Dirichlet nodes
    none; pressure rows only among poroelastic subdomains, Dirichlet on x = 0, x = 1, y = 0."""
    k = case.order_k
    cx, cy = np.asarray(case.cells_x), np.asarray(case.cells_y)
    ox, oy = np.concatenate([[0], np.cumsum(cx)]), np.concatenate([[0], np.cumsum(cy)])
    mu = np.zeros((k * oy[-1] + 1, k * ox[-1] + 1), dtype=np.int64)
    mp = np.zeros((oy[case.poro_rows] + 1, ox[-1] + 1), dtype=np.int64)
    for j in range(case.nsub_y):
        for i in range(case.nsub_x):
            mu[k * oy[j]: k * oy[j + 1] + 1, k * ox[i]: k * ox[i + 1] + 1] += 1
            if j < case.poro_rows:
                mp[oy[j]: oy[j + 1] + 1, ox[i]: ox[i + 1] + 1] += 1
    n_u = 2 * int(np.maximum(mu[1:-1, 1:-1] - 1, 0).sum())
    n_p = int(np.maximum(mp[1:, 1:-1] - 1, 0).sum())
    n_float = max(case.nsub_x - 2, 0) * max(case.nsub_y - 2, 0)
    return n_u + n_p, n_p, n_float


def test_brute_force_count_agrees_with_oracle_on_small_cases():
    from oracle.monolithic import Discretization
    for case in SMALL:
        d = Discretization(case)
        assert _brute_force_counts(case)[:2] == (d.iface.n_lambda, int(d.iface.is_p.sum())), case.name


@pytest.mark.parametrize("make", [W.config2, W.config3], ids=["8x8 x 32^2 P2", "32x32 uneven 16..48 P2"])
def test_plan_counts_brute_force(make):
    case = make()
    s = F.plan(case)
    n_lambda, n_lambda_p, n_float = _brute_force_counts(case)
    assert (s.n_lambda, s.n_lambda_p, s.n_floating) == (n_lambda, n_lambda_p, n_float)


def test_plan_config5_closed_form():
    """64 x 64 subdomains of 24 x 24 P2 cells, lower half poroelastic.  Displacement: 63
    vertical and 63 horizontal interface lines of 64 * 48 - 1 interior nodes, 63^2 four-way
    cross points (3 rows per component), every other line node 1 row.  Pressure: 63 vertical
    lines of 32 * 24 nodes above y = 0 (the y = 1/2 end is a no-flux, not a Dirichlet, node),
    31 horizontal lines of 64 * 24 - 1 nodes, 63 * 31 cross points."""
    case = W.config5()
    s = F.plan(case)
    cross_u = 63 * 63
    line_u = 2 * 63 * (64 * 48 - 1) - 2 * cross_u
    n_u = 2 * (line_u + 3 * cross_u)
    cross_p = 63 * 31
    n_p = (63 * 32 * 24 - cross_p) + (31 * (64 * 24 - 1) - cross_p) + 3 * cross_p
    assert (n_u, n_p) == (781830, 97922)
    assert s.n_lambda == n_u + n_p and s.n_lambda_p == n_p
    assert s.n_floating == 62 * 62 and s.nsub == 4096
    assert s.n_unode_total == 4096 * 49 * 49 and s.n_pnode_total == 4096 * 25 * 25
    s64 = F.plan(case, precision="fp64")
    assert s64.factor_bytes == 2 * s.factor_bytes and s64.n_dofs == s.n_dofs


def test_plan_rejects_what_create_rejects():
    for bad in (W.small_case(2, 2, 4).with_(order_k=3), W.small_case(2, 2, 4).with_(tol=0.0),
                W.small_case(2, 2, 4).with_(source="point", src_node=(4, 2))):
        with pytest.raises(F.FetipeError) as e:
            F.plan(bad)
        assert e.value.status == F.FP_ERR_INVALID
