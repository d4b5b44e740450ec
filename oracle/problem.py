"""Problem data (test infrastructure; see ``oracle/__init__``).

* Multiphysics constants kappa_1..3 of Sec. 2.2 (Eq. (2.17) ff.).
* Lame constants from (E, nu): lambda = E nu / ((1+nu)(1-2nu)); the paper's Table 2
  prints mu = E / (1+nu), which is not the standard E / (2(1+nu)); both are offered
  (``mu_convention``), the paper's one only to compare with its tables.
* Test Case 1 (Sec. 4.1): u_P = (sin 2pi x sin 2pi y) (1, 1), p = sin pi x sin pi y,
  u_E = u_P + (0, -alpha p (y - 1/2) / (lambda + 2 mu)); the sources are derived here by
  hand from Eqs. (2.1)-(2.3) (stationary solution: the time derivative vanishes) and are
  pinned by tests/test_oracle_problem.py against central finite differences of the
  closed forms, and against the transmission conditions (2.12)-(2.14).
* Barry-Mercer-type data of Sec. 4.3 and the point fluid source z = q(t) delta(x - x_s).
* Time-dependent variant ``manufactured_t``: the same closed form times g(t) = 1 + t.
  Backward Euler is exact in time for it (the time derivative is constant), and every
  source is the stationary one times g(t), except z, which gains g'(t) eta:
  z(t) = g(t) z_s + g'(t) (c0 p_s + alpha div u_s).
"""
import numpy as np

PI = np.pi


def lame_from_young(E, nu, mu_convention="standard"):
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (1.0 + nu) if mu_convention == "paper" else E / (2.0 * (1.0 + nu))
    return lam, mu


def kappas(alpha, c0, lam):
    """kappa_1, kappa_2, kappa_3 of Sec. 2.2."""
    den = alpha * alpha + c0 * lam
    return alpha / den, lam / den, c0 / den


class Manufactured:
    """Closed-form solution and sources of Test Case 1 (Sec. 4.1)."""

    def __init__(self, lam, mu, alpha, c0, K=1.0, mu_f=1.0):
        self.lam, self.mu, self.alpha, self.c0, self.K, self.mu_f = lam, mu, alpha, c0, K, mu_f
        self.beta = alpha / (lam + 2.0 * mu)

    # closed forms -----------------------------------------------------------------
    @staticmethod
    def _s(x, y):
        return np.sin(2 * PI * x) * np.sin(2 * PI * y)

    @staticmethod
    def _c(x, y):
        return np.cos(2 * PI * x) * np.cos(2 * PI * y)

    @staticmethod
    def q(x, y):
        return np.sin(PI * x) * np.sin(PI * y)

    def u_P(self, x, y):
        s = self._s(x, y)
        return s, s

    def p(self, x, y):
        return self.q(x, y)

    def g(self, x, y):
        """Second component of u_E - u_P."""
        return -self.beta * self.q(x, y) * (y - 0.5)

    def u_E(self, x, y):
        s = self._s(x, y)
        return s, s + self.g(x, y)

    def div_u_P(self, x, y):
        return 2 * PI * (np.cos(2 * PI * x) * np.sin(2 * PI * y)
                         + np.sin(2 * PI * x) * np.cos(2 * PI * y))

    def div_u_E(self, x, y):
        qy = PI * np.sin(PI * x) * np.cos(PI * y)
        g_y = -self.beta * (qy * (y - 0.5) + self.q(x, y))
        return self.div_u_P(x, y) + g_y

    def xi_P(self, x, y):
        return self.alpha * self.p(x, y) - self.lam * self.div_u_P(x, y)

    def xi_E(self, x, y):
        return -self.lam * self.div_u_E(x, y)

    def eta(self, x, y):
        # Eq. (2.17): eta = c0 p + alpha div u  (reading of the sign clash at Eq. (2.33))
        return self.c0 * self.p(x, y) + self.alpha * self.div_u_P(x, y)

    # sources ----------------------------------------------------------------------
    def _minus_div_sigma_uP(self, x, y):
        s, c = self._s(x, y), self._c(x, y)
        v = 8 * PI ** 2 * self.mu * s - 4 * PI ** 2 * (self.lam + self.mu) * (c - s)
        return v, v

    def f_P(self, x, y):
        """-div sigma(u_P) + alpha grad p  (Eq. (2.1))."""
        a, b = self._minus_div_sigma_uP(x, y)
        px = PI * np.cos(PI * x) * np.sin(PI * y)
        py = PI * np.sin(PI * x) * np.cos(PI * y)
        return a + self.alpha * px, b + self.alpha * py

    def f_E(self, x, y):
        """-div sigma(u_E)  (Eq. (2.3))."""
        a, b = self._minus_div_sigma_uP(x, y)
        q = self.q(x, y)
        qx = PI * np.cos(PI * x) * np.sin(PI * y)
        qy = PI * np.sin(PI * x) * np.cos(PI * y)
        qxy = PI ** 2 * np.cos(PI * x) * np.cos(PI * y)
        bt, ym = self.beta, (y - 0.5)
        g_xy = -bt * (qxy * ym + qx)
        g_yy = bt * PI ** 2 * q * ym - 2 * bt * qy
        lap_g = 2 * bt * PI ** 2 * q * ym - 2 * bt * qy
        lm = self.lam + self.mu
        return a - lm * g_xy, b - self.mu * lap_g - lm * g_yy

    def z(self, x, y):
        """-div((K/mu_f) grad p) for the stationary solution (Eq. (2.2))."""
        return (self.K / self.mu_f) * 2 * PI ** 2 * self.q(x, y)

    def traction_on_interface(self, x):
        """lambda = sigma_E(u_E) . n_{E->P} at y = 1/2 (Eq. (2.27))."""
        a = 2 * PI * self.mu * np.sin(2 * PI * x)
        b = 2 * PI * (self.lam + 2 * self.mu) * np.sin(2 * PI * x) + self.alpha * np.sin(PI * x)
        return a, b


def time_factor(t):
    """g(t) = 1 + t and g'(t) = 1 of the time-dependent manufactured variant."""
    return 1.0 + t, 1.0


def barry_mercer_p2(x, t):
    """Pressure data on Gamma_2 (Sec. 4.3): sin t on 0.2 <= x <= 0.8, else 0."""
    return np.where((x >= 0.2) & (x <= 0.8), np.sin(t), 0.0)


def point_source_q(case, t):
    """Strength q(t) = sin(omega t) of the point fluid source."""
    return np.sin(case.q_omega * t)
