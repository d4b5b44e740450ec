"""Pins of the oracle's point fluid source (Sec. 4.3's Barry-Mercer-type test with the fluid
source z = q(t) delta(x - x_s), q(t) = sin(omega t), at a P1 vertex x_s).

* The load: the nodal source vector (z, phi_i) of a Dirac at a vertex is q(t) at that vertex
  and zero elsewhere (P1 basis functions are 1 at their own vertex and 0 at the others), so it
  sits at one node of one poroelastic subdomain and sums to q(t).
* The sign and the tau factor, through the fluid balance of Eq. (2.2) (mass conservation:
  d eta / dt - div(K grad p) = z): starting from zero, one backward-Euler step adds
  tau q(t_1) of fluid content at the source, part of which drains through the p = 0 boundary
  in the same step, so the total content (eta^1, 1) = 1^T R eta^1 has the sign of q and lies in
  (0, tau q] -- close to tau q for a short step.  A dropped tau, a flipped sign or a wrong
  node breaks it.  The pressure peaks at the source with the sign of q."""
import numpy as np
import pytest

from oracle.monolithic import Discretization, solve_monolithic
from paper_2509_06673_gb300 import workloads as W

SRC = (6, 5)   # global P1 indices: inside subdomain (1, 1) of 4 x 4 subdomains of 4 x 4 cells


def _case(q_omega, tau):
    return W.small_case(4, 4, 4, k=2, lame_lambda=9.0, tau=tau, n_steps=1, source="point", src_node=SRC,
                        q_omega=q_omega)


@pytest.mark.parametrize("t", [0.01, 0.037])
def test_point_load_is_q_at_one_vertex(t):
    case = _case(30.0, 1e-2)
    d = Discretization(case)
    q = np.sin(case.q_omega * t)
    owners = []
    total = 0.0
    for s, L in enumerate(d.locals):
        if not L.m.is_poro:
            continue
        zero = np.zeros(L.m.n_pnode)
        b = L.rhs(t, zero)
        # p-rows: -R eta^{n-1} - tau Z (+ lifting of p = 0, which is zero): Z on free nodes
        Z = -b[L.off_p:] / case.tau
        nz = np.flatnonzero(np.abs(Z) > 1e-300)
        if nz.size:
            owners.append((s, nz))
            total += Z.sum()
            node = L.pfree[nz[0]]
            i, j = L.m.i0 + node % L.m.npx, L.m.j0 + node // L.m.npx
            assert (i, j) == SRC
    assert len(owners) == 1 and owners[0][1].size == 1
    assert owners[0][0] == 1 * 4 + 1 and case.is_poro(owners[0][0])
    assert total == pytest.approx(q, rel=1e-14)


@pytest.mark.parametrize("phase", [0.3, 4.5])   # omega tau: q(t_1) = sin(omega tau) > 0 and < 0
@pytest.mark.parametrize("tau", [1e-2, 1e-3])
def test_point_source_fluid_balance(phase, tau):
    q_omega = phase / tau
    case = _case(q_omega, tau)
    d = Discretization(case)
    step = solve_monolithic(case, d)[0]
    q = np.sin(q_omega * tau)
    content = sum(float(np.asarray(L.R_full.sum(axis=0)).ravel() @ step["fields"][s][2])
                  for s, L in enumerate(d.locals) if L.m.is_poro)
    ratio = content / (tau * q)
    assert 0.5 < ratio <= 1.0 + 1e-9, ratio
    p_all = [(s, f[3]) for s, f in enumerate(step["fields"]) if f[3] is not None]
    s_src = 1 * 4 + 1
    L = d.locals[s_src]
    k = L.point_node()
    p_src = step["fields"][s_src][3][k]
    assert np.sign(p_src) == np.sign(q)
    assert abs(p_src) == max(np.abs(p).max() for _, p in p_all)
