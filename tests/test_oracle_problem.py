"""Pins of the closed-form data of Test Case 1 against finite differences and Sec. 2."""
import numpy as np
import pytest

from oracle.problem import Manufactured, kappas, lame_from_young

H = 1e-4


def _grad(f, x, y):
    return ((f(x + H, y) - f(x - H, y)) / (2 * H), (f(x, y + H) - f(x, y - H)) / (2 * H))


def _stress(mf, ufun, x, y, lam, mu):
    """sigma(u) by central differences: returns s11, s12, s22."""
    u1 = lambda a, b: ufun(a, b)[0]
    u2 = lambda a, b: ufun(a, b)[1]
    u1x, u1y = _grad(u1, x, y)
    u2x, u2y = _grad(u2, x, y)
    div = u1x + u2y
    return (2 * mu * u1x + lam * div, mu * (u1y + u2x), 2 * mu * u2y + lam * div)


def _neg_div_stress(mf, ufun, x, y, lam, mu):
    s = lambda a, b: _stress(mf, ufun, a, b, lam, mu)
    s11x = (s(x + H, y)[0] - s(x - H, y)[0]) / (2 * H)
    s12y = (s(x, y + H)[1] - s(x, y - H)[1]) / (2 * H)
    s12x = (s(x + H, y)[1] - s(x - H, y)[1]) / (2 * H)
    s22y = (s(x, y + H)[2] - s(x, y - H)[2]) / (2 * H)
    return -(s11x + s12y), -(s12x + s22y)


@pytest.mark.parametrize("lam,mu,alpha,c0", [(1.0, 1.0, 1.0, 1.0), (49.0, 1.0, 0.7, 0.3)])
def test_sources_match_finite_differences(lam, mu, alpha, c0):
    mf = Manufactured(lam, mu, alpha, c0, K=2.0, mu_f=0.5)
    rng = np.random.default_rng(0)
    for x, y in rng.uniform(0.05, 0.95, size=(6, 2)):
        a, b = _neg_div_stress(mf, mf.u_P, x, y, lam, mu)
        px, py = _grad(mf.p, x, y)
        fx, fy = mf.f_P(x, y)
        scale = 1 + abs(lam)
        assert abs(a + alpha * px - fx) < 2e-4 * scale and abs(b + alpha * py - fy) < 2e-4 * scale
        a, b = _neg_div_stress(mf, mf.u_E, x, y, lam, mu)
        fx, fy = mf.f_E(x, y)
        assert abs(a - fx) < 2e-4 * scale and abs(b - fy) < 2e-4 * scale
        lap = ((mf.p(x + H, y) - 2 * mf.p(x, y) + mf.p(x - H, y))
               + (mf.p(x, y + H) - 2 * mf.p(x, y) + mf.p(x, y - H))) / H ** 2
        assert abs(-(2.0 / 0.5) * lap - mf.z(x, y)) < 1e-4 * 40
        # multiphysics variables of Sec. 2.2
        ux, uy = _grad(lambda a, b: mf.u_P(a, b)[0], x, y)
        vx, vy = _grad(lambda a, b: mf.u_P(a, b)[1], x, y)
        div = ux + vy
        assert abs(mf.div_u_P(x, y) - div) < 1e-6
        assert abs(mf.xi_P(x, y) - (alpha * mf.p(x, y) - lam * div)) < 1e-5 * scale
        assert abs(mf.eta(x, y) - (c0 * mf.p(x, y) + alpha * div)) < 1e-6


@pytest.mark.parametrize("lam,mu,alpha", [(1.0, 1.0, 1.0), (499.0, 1.0, 1.0)])
def test_transmission_conditions(lam, mu, alpha):
    """Eqs. (2.12)-(2.14) at y = 1/2 and the multiplier of Eq. (2.27)."""
    mf = Manufactured(lam, mu, alpha, 1.0)
    for x in np.linspace(0.05, 0.95, 7):
        y = 0.5
        assert np.allclose(mf.u_P(x, y), mf.u_E(x, y), atol=1e-14)
        sP = _stress(mf, mf.u_P, x, y, lam, mu)
        sE = _stress(mf, mf.u_E, x, y, lam, mu)
        p = mf.p(x, y)
        # total stress of P times n_{P->E} = (0, 1), equal to sigma_E times (0, 1)
        tP = np.array([sP[1], sP[2] - alpha * p])
        tE = np.array([sE[1], sE[2]])
        assert np.allclose(tP, tE, atol=2e-5 * (1 + lam))
        # lambda = sigma_E(u_E) n_{E->P}
        assert np.allclose(-tE, mf.traction_on_interface(x), atol=2e-5 * (1 + lam))
        assert abs(_grad(mf.p, x, y)[1]) < 1e-8  # no flux


def test_kappa_identities():
    for alpha, c0, lam in ((1.0, 1.0, 1.0), (0.8, 0.1, 499.0), (1.0, 1e-3, 2777.0)):
        k1, k2, k3 = kappas(alpha, c0, lam)
        assert abs(k1 * k1 + k2 * k3 - 1.0 / (alpha * alpha + c0 * lam)) < 1e-14
        assert abs(k3 + k1 * k1 / k2 - 1.0 / lam) < 1e-14 / min(lam, 1)
        # p = k1 xi + k2 eta inverts Eq. (2.17); for div u the derivation gives
        # div u = k1 eta - k3 xi as in Eq. (2.20), not k3 xi - k1 eta as printed after (2.17)
        p, div = 0.37, -1.3
        xi = alpha * p - lam * div
        eta = c0 * p + alpha * div
        assert abs(k1 * xi + k2 * eta - p) < 1e-12
        assert abs(k1 * eta - k3 * xi - div) < 1e-12
        assert abs(k3 * xi - k1 * eta - div) > 1.0


def test_lame():
    lam, mu = lame_from_young(1e4, 0.2)
    assert abs(lam - 1e4 * 0.2 / (1.2 * 0.6)) < 1e-9 and abs(mu - 1e4 / 2.4) < 1e-9
    assert abs(lame_from_young(1e4, 0.2, "paper")[1] - 1e4 / 1.2) < 1e-9
