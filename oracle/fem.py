"""Element matrices of the bilinear forms (test infrastructure; see ``oracle/__init__``).

Sec. 2.3, Eqs. (2.21)-(2.23):
    a_D(u, v) = 2 mu (eps(u), eps(v)),     b_D(v, xi) = -(xi, div v),
    a_f(p, q) = (1/mu_f) (K grad p, grad q),
plus the P1 mass matrix R (Sec. 2.5).  Displacements use P_k (k = 1, 2), scalars P1
(Sec. 2.4).  Every integrand here is a polynomial of degree <= 2 on an affine triangle,
so ``collapsed_gauss(3)`` (exact to degree 4) integrates it exactly.  Loads use
``radon7`` (Sec. 4.1 does not name a rule).

Local displacement dof order inside an element: node-major, (x, y) per node.
P2 local nodes: vertices a, b, c, then midpoints (a,b), (b,c), (c,a).

Pinned by tests/test_oracle_fem.py: rigid modes annihilated by a_D and b_D, mass sums to
the area, a_D of a linear field against its closed form, b_D against -(xi, div v) of
polynomials integrated in closed form, symmetry, patch test.
"""
import numpy as np

from .quadrature import collapsed_gauss, radon7


def bary_grads(xy):
    """Gradients of the barycentric coordinates and areas.  xy: (ne, 3, 2)."""
    a, b, c = xy[:, 0], xy[:, 1], xy[:, 2]
    J = np.stack([b - a, c - a], axis=-1)          # (ne, 2, 2) columns b-a, c-a
    det = J[:, 0, 0] * J[:, 1, 1] - J[:, 0, 1] * J[:, 1, 0]
    Jinv = np.stack([np.stack([J[:, 1, 1], -J[:, 0, 1]], -1),
                     np.stack([-J[:, 1, 0], J[:, 0, 0]], -1)], 1) / det[:, None, None]
    # reference gradients of (l_a, l_b, l_c) w.r.t. (xi, eta)
    gref = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]])
    G = np.einsum("ij,ejk->eik", gref, Jinv)        # grad l_i = J^{-T} gref_i
    return G, 0.5 * np.abs(det)


def shape(k, lam):
    """Basis values at barycentric points lam (nq, 3) -> (nq, nloc)."""
    l0, l1, l2 = lam[:, 0], lam[:, 1], lam[:, 2]
    if k == 1:
        return np.stack([l0, l1, l2], axis=-1)
    return np.stack([l0 * (2 * l0 - 1), l1 * (2 * l1 - 1), l2 * (2 * l2 - 1),
                     4 * l0 * l1, 4 * l1 * l2, 4 * l2 * l0], axis=-1)


def shape_grad(k, lam, G):
    """Basis gradients: lam (nq, 3), G (ne, 3, 2) -> (ne, nq, nloc, 2)."""
    ne, nq = G.shape[0], lam.shape[0]
    if k == 1:
        return np.broadcast_to(G[:, None, :, :], (ne, nq, 3, 2)).copy()
    L = lam[None, :, :, None]        # (1, nq, 3, 1)
    Gv = G[:, None, :, :]            # (ne, 1, 3, 2)
    out = np.empty((ne, nq, 6, 2))
    out[:, :, 0:3, :] = (4 * L - 1) * Gv
    for m, (i, j) in enumerate(((0, 1), (1, 2), (2, 0))):
        out[:, :, 3 + m, :] = 4 * (L[:, :, i] * Gv[:, :, j] + L[:, :, j] * Gv[:, :, i])
    return out


def _vector_strain(dphi):
    """Strain tensors of the vector basis phi_i e_c.  dphi (ne, nq, n, 2) ->
    eps (ne, nq, 2n, 2, 2) with dof index 2*i + c, and div (ne, nq, 2n)."""
    ne, nq, n, _ = dphi.shape
    eps = np.zeros((ne, nq, 2 * n, 2, 2))
    div = np.zeros((ne, nq, 2 * n))
    px, py = dphi[..., 0], dphi[..., 1]
    # phi e_x: eps = [[phi_x, phi_y/2], [phi_y/2, 0]], div = phi_x
    eps[:, :, 0::2, 0, 0] = px
    eps[:, :, 0::2, 0, 1] = 0.5 * py
    eps[:, :, 0::2, 1, 0] = 0.5 * py
    div[:, :, 0::2] = px
    # phi e_y: eps = [[0, phi_x/2], [phi_x/2, phi_y]], div = phi_y
    eps[:, :, 1::2, 0, 1] = 0.5 * px
    eps[:, :, 1::2, 1, 0] = 0.5 * px
    eps[:, :, 1::2, 1, 1] = py
    div[:, :, 1::2] = py
    return eps, div


def element_matrices(xy, k, mu, perm=None, mu_f=1.0):
    """Element matrices on triangles xy (ne, 3, 2).

    Returns A (ne, 2n, 2n) of a_D, Bd (ne, 3, 2n) with [Bd]_{ij} = b_D(theta_j, phi_i),
    R (ne, 3, 3) mass, Af (ne, 3, 3) of a_f with per-element scalar permeability.
    """
    lam, w = collapsed_gauss(3)
    G, area = bary_grads(xy)
    dphi = shape_grad(k, lam, G)
    eps, div = _vector_strain(dphi)
    wa = w[None, :] * area[:, None]                         # (ne, nq)
    A = 2.0 * mu * np.einsum("eq,eqiab,eqjab->eij", wa, eps, eps)
    phi1 = shape(1, lam)                                    # (nq, 3)
    Bd = -np.einsum("eq,qi,eqj->eij", wa, phi1, div)
    R = np.einsum("eq,qi,qj->eij", wa, phi1, phi1)
    K = np.ones(xy.shape[0]) if perm is None else np.asarray(perm, dtype=float)
    Af = (K / mu_f)[:, None, None] * area[:, None, None] * np.einsum("eia,eja->eij", G, G)
    return A, Bd, R, Af


def map_points(xy, lam):
    """Physical coordinates of barycentric points: (ne, nq, 2)."""
    return np.einsum("qc,ecd->eqd", lam, xy)


def load_vector_u(xy, k, f):
    """(f, theta_i) per element with the degree-5 rule; f(x, y) -> (fx, fy)."""
    lam, w = radon7()
    _, area = bary_grads(xy)
    X = map_points(xy, lam)
    fx, fy = f(X[..., 0], X[..., 1])
    phi = shape(k, lam)                                     # (nq, n)
    wa = w[None, :] * area[:, None]
    out = np.zeros((xy.shape[0], 2 * phi.shape[1]))
    out[:, 0::2] = np.einsum("eq,eq,qi->ei", wa, fx, phi)
    out[:, 1::2] = np.einsum("eq,eq,qi->ei", wa, fy, phi)
    return out


def load_vector_s(xy, g):
    """(g, phi_i) for P1 phi with the degree-5 rule."""
    lam, w = radon7()
    _, area = bary_grads(xy)
    X = map_points(xy, lam)
    gv = g(X[..., 0], X[..., 1])
    wa = w[None, :] * area[:, None]
    return np.einsum("eq,eq,qi->ei", wa, gv, shape(1, lam))
