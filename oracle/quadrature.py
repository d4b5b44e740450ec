"""Quadrature on triangles (test infrastructure; see ``oracle/__init__``).

Rules are returned in barycentric coordinates with weights normalised to sum to 1, so
that the integral over a triangle T is ``area(T) * sum_q w_q f(x_q)``.

* ``radon7`` -- the 7-point symmetric rule of degree 5 (Radon 1948; Stroud's T2:5-1).
  The paper does not name its quadrature (Sec. 4.1 is silent); this rule is the load rule
  of the whole project and the CUDA path evaluates the same published rule from its own
  closed form.  Pinned by exactness on all monomials of degree <= 5 and inexactness at 6.
* ``collapsed_gauss(n)`` -- conical-product Gauss-Legendre rule, exact to total degree
  2n-2; used for element matrices (degree 2 integrands) and for error norms.
  Pinned by monomial exactness.
"""
import numpy as np


def radon7():
    s15 = np.sqrt(15.0)
    pts = [(1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0)]
    wts = [9.0 / 40.0]
    for a, w in (((6.0 - s15) / 21.0, (155.0 - s15) / 1200.0),
                 ((6.0 + s15) / 21.0, (155.0 + s15) / 1200.0)):
        b = 1.0 - 2.0 * a
        pts += [(b, a, a), (a, b, a), (a, a, b)]
        wts += [w, w, w]
    return np.array(pts), np.array(wts)


def collapsed_gauss(n):
    x, w = np.polynomial.legendre.leggauss(n)
    s = 0.5 * (x + 1.0)
    ws = 0.5 * w
    pts, wts = [], []
    for i in range(n):
        for j in range(n):
            xi = s[i]
            eta = (1.0 - s[i]) * s[j]
            pts.append((1.0 - xi - eta, xi, eta))
            # reference triangle has area 1/2: normalise so the weights sum to 1
            wts.append(2.0 * ws[i] * ws[j] * (1.0 - s[i]))
    return np.array(pts), np.array(wts)
