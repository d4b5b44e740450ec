"""Pins of the oracle's quadrature, mesh and element matrices against closed forms."""
import math

import numpy as np
import pytest

from oracle import fem
from oracle.quadrature import radon7, collapsed_gauss
from oracle.mesh import build_meshes
from paper_2509_06673_gb300 import workloads as W


def _mono_exact(a, b):
    # integral over the reference triangle of xi^a eta^b = a! b! / (a+b+2)!
    return math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)


def _quad_ref(rule, a, b):
    lam, w = rule
    xi, eta = lam[:, 1], lam[:, 2]
    return 0.5 * np.sum(w * xi ** a * eta ** b)


def test_radon7_degree5():
    r = radon7()
    assert abs(r[1].sum() - 1.0) < 1e-15
    for d in range(6):
        for a in range(d + 1):
            assert abs(_quad_ref(r, a, d - a) - _mono_exact(a, d - a)) < 1e-15
    errs = [abs(_quad_ref(r, a, 6 - a) - _mono_exact(a, 6 - a)) for a in range(7)]
    assert max(errs) > 1e-6  # degree exactly 5


@pytest.mark.parametrize("n", [2, 3, 6])
def test_collapsed_gauss_degree(n):
    r = collapsed_gauss(n)
    for d in range(2 * n - 1):
        for a in range(d + 1):
            assert abs(_quad_ref(r, a, d - a) - _mono_exact(a, d - a)) < 1e-14


def _tri():
    return np.array([[[0.1, 0.2], [0.9, 0.35], [0.3, 0.8]]])


def _area(t):
    (ax, ay), (bx, by), (cx, cy) = t
    return 0.5 * abs((bx - ax) * (cy - ay) - (by - ay) * (cx - ax))


@pytest.mark.parametrize("k", [1, 2])
def test_rigid_modes_annihilated(k):
    xy = _tri()
    A, Bd, R, Af = fem.element_matrices(xy, k, mu=1.7)
    lam = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [.5, .5, 0], [0, .5, .5], [.5, 0, .5]])[: 3 * k]
    nodes = lam @ xy[0]
    for mode in (lambda x, y: (1.0, 0.0), lambda x, y: (0.0, 1.0), lambda x, y: (-y, x)):
        v = np.zeros(2 * nodes.shape[0])
        for i, (x, y) in enumerate(nodes):
            v[2 * i], v[2 * i + 1] = mode(x, y)
        assert np.abs(A[0] @ v).max() < 1e-12
        assert np.abs(Bd[0] @ v).max() < 1e-12
    assert abs(R[0].sum() - _area(xy[0])) < 1e-15
    assert np.abs(Af[0] @ np.ones(3)).max() < 1e-13
    assert np.allclose(A[0], A[0].T) and np.allclose(R[0], R[0].T) and np.allclose(Af[0], Af[0].T)


@pytest.mark.parametrize("k", [1, 2])
def test_linear_field_energy_and_divergence(k):
    """a(u, v) = 2 mu area eps(u):eps(v) and b(u, phi_i) = -div u * area / 3 for linear fields."""
    xy = _tri()
    mu = 0.8
    A, Bd, R, Af = fem.element_matrices(xy, k, mu=mu)
    area = _area(xy[0])
    lam = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [.5, .5, 0], [0, .5, .5], [.5, 0, .5]])[: 3 * k]
    nodes = lam @ xy[0]
    rng = np.random.default_rng(1)
    G1, G2 = rng.normal(size=(2, 2)), rng.normal(size=(2, 2))

    def interp(G):
        v = np.zeros(2 * nodes.shape[0])
        for i, x in enumerate(nodes):
            v[2 * i: 2 * i + 2] = G @ x
        return v
    e1, e2 = 0.5 * (G1 + G1.T), 0.5 * (G2 + G2.T)
    assert abs(interp(G1) @ A[0] @ interp(G2) - 2 * mu * area * np.sum(e1 * e2)) < 1e-12
    assert np.allclose(Bd[0] @ interp(G1), -np.trace(G1) * area / 3.0, atol=1e-13)
    # a_f of linear scalars: area * grad p . grad q
    g1, g2 = rng.normal(size=2), rng.normal(size=2)
    p1, p2 = xy[0] @ g1, xy[0] @ g2
    assert abs(p1 @ Af[0] @ p2 - area * g1 @ g2) < 1e-12


def test_p2_reproduces_quadratics():
    xy = _tri()
    lam, _ = radon7()
    phi = fem.shape(2, lam)
    nodes = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [.5, .5, 0], [0, .5, .5], [.5, 0, .5]]) @ xy[0]
    f = lambda x, y: 1 + 2 * x - y + 3 * x * x - x * y + 0.5 * y * y
    X = fem.map_points(xy, lam)[0]
    assert np.allclose(phi @ f(nodes[:, 0], nodes[:, 1]), f(X[:, 0], X[:, 1]), atol=1e-13)
    assert np.allclose(phi.sum(axis=1), 1.0)


def test_mesh_partition_matches():
    c = W.grid_case("t", 3, 2, [2, 3, 4], [3, 2], order_k=2)
    ms = build_meshes(c)
    total = sum(fem.bary_grads(m.elem_xy)[1].sum() for m in ms)
    assert abs(total - 1.0) < 1e-13
    coords = {}
    for m in ms:
        x, y = m.unode_xy()
        for a in range(m.n_unode):
            key = m.unode_key(a)
            if key in coords:
                assert np.allclose(coords[key], (x[a], y[a]), atol=1e-14)
            coords[key] = (x[a], y[a])
    assert len(coords) == (2 * 9 + 1) * (2 * 5 + 1)
