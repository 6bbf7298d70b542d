"""Closed-form solutions used to pin the oracle (test infrastructure only).

* Manufactured 2-D solution (paper §Poroelasticity strong form, data chosen so
  that every term is exercised):  u = (S t, S t), p = C t with
  S = sin(pi x) sin(pi y), C = cos(pi x) cos(pi y), q = -(K/eta) grad p,
  rho_f g = 0.  The loads below were derived by hand from the strong form and
  are cross-checked symbolically in the tests.
* Space-exact manufactured solution for time-order studies: u = (P(x,y) g(t), 0)
  with P = x(1-x)y(1-y) in Q2, p = (x + 2y) g(t) in DGQ1, q = -(K/eta) grad p in RT1.
* Terzaghi one-dimensional consolidation: drained loaded top, undrained rigid
  bottom, series solution of the pressure diffusion equation.
"""
from __future__ import annotations

import numpy as np

PI = np.pi


class MMS2D:
    """u = (S t, S t), p = C t on the unit square; Dirichlet u, natural p."""

    def __init__(self, lam, mu, b, invM, eta, K):
        self.lam, self.mu, self.b, self.invM, self.eta, self.K = lam, mu, b, invM, eta, K

    def u(self, X, t):
        s = np.sin(PI * X[:, 0]) * np.sin(PI * X[:, 1])
        return np.stack([s * t, s * t], axis=1)

    def p(self, X, t):
        return np.cos(PI * X[:, 0]) * np.cos(PI * X[:, 1]) * t

    def q(self, X, t):
        k = self.K / self.eta
        return np.stack([k * PI * np.sin(PI * X[:, 0]) * np.cos(PI * X[:, 1]) * t,
                         k * PI * np.cos(PI * X[:, 0]) * np.sin(PI * X[:, 1]) * t], axis=1)

    def body_force(self, X, t):
        """rho_b g = -div(2 mu eps(u) + lam div u I - b p I)
                   = -mu lap u - (mu+lam) grad div u + b grad p."""
        x, y = X[:, 0], X[:, 1]
        mu, lam, b = self.mu, self.lam, self.b
        s = np.sin(PI * x) * np.sin(PI * y)
        cxy = np.cos(PI * (x + y))
        fx = 2 * mu * PI ** 2 * s - (mu + lam) * PI ** 2 * cxy - b * PI * np.sin(PI * x) * np.cos(PI * y)
        fy = 2 * mu * PI ** 2 * s - (mu + lam) * PI ** 2 * cxy - b * PI * np.cos(PI * x) * np.sin(PI * y)
        return np.stack([fx * t, fy * t], axis=1)

    def source(self, X, t):
        """f = b d_t div u + (1/M) d_t p + div q."""
        x, y = X[:, 0], X[:, 1]
        C = np.cos(PI * x) * np.cos(PI * y)
        return self.b * PI * np.sin(PI * (x + y)) + self.invM * C + 2 * PI ** 2 * (self.K / self.eta) * C * t

    def p_boundary(self, X, t, face):
        return self.p(X, t)


class PolyMMS2D:
    """Space-exact manufactured solution with a time profile g(t) = sin(omega t) + 1 - cos(omega t)
    (not polynomial, so the dG(r) time error is visible):
    u = (P g, 0), P = x(1-x) y(1-y);  p = (x + 2y) g;  q = -(K/eta)(1, 2) g."""

    def __init__(self, lam, mu, b, invM, eta, K, omega=3.0):
        self.lam, self.mu, self.b, self.invM, self.eta, self.K, self.om = lam, mu, b, invM, eta, K, omega

    def g(self, t):
        return np.sin(self.om * t) + 1.0 - np.cos(self.om * t)

    def dg(self, t):
        return self.om * (np.cos(self.om * t) + np.sin(self.om * t))

    def u(self, X, t):
        x, y = X[:, 0], X[:, 1]
        P = x * (1 - x) * y * (1 - y)
        return np.stack([P * self.g(t), 0 * P], axis=1)

    def p(self, X, t):
        return (X[:, 0] + 2 * X[:, 1]) * self.g(t)

    def q(self, X, t):
        k = self.K / self.eta
        one = np.ones(len(X))
        return np.stack([-k * one * self.g(t), -2 * k * one * self.g(t)], axis=1)

    def body_force(self, X, t):
        """-mu lap u - (mu+lam) grad div u + b grad p for u = (P, 0)."""
        x, y = X[:, 0], X[:, 1]
        mu, lam, b = self.mu, self.lam, self.b
        Pxx = -2 * y * (1 - y)
        Pyy = -2 * x * (1 - x)
        Pxy = (1 - 2 * x) * (1 - 2 * y)
        lapx = Pxx + Pyy
        # div u = P_x g ; grad div u = (P_xx, P_xy) g ; grad p = (1, 2) g
        gt = self.g(t)
        fx = (-mu * lapx - (mu + lam) * Pxx + b) * gt
        fy = (-(mu + lam) * Pxy + 2 * b) * gt
        return np.stack([fx, fy], axis=1)

    def source(self, X, t):
        """b d_t div u + (1/M) d_t p + div q, div q = 0."""
        x, y = X[:, 0], X[:, 1]
        Px = (1 - 2 * x) * y * (1 - y)
        return (self.b * Px + self.invM * (x + 2 * y)) * self.dg(t)

    def p_boundary(self, X, t, face):
        return self.p(X, t)


def terzaghi_p0(lam, mu, b, invM, load=1.0):
    """Undrained pressure after a sudden load: b S / (b^2 + (lam + 2 mu) / M)."""
    return b * load / (b * b + (lam + 2 * mu) * invM)


def terzaghi_c(lam, mu, b, invM, K, eta):
    """Consolidation coefficient (K/eta) / (1/M + b^2/(lam + 2 mu))."""
    return (K / eta) / (invM + b * b / (lam + 2 * mu))


def terzaghi_pressure(z, t, lam, mu, b, invM, K, eta, H=1.0, load=1.0, terms=400):
    """p(z, t) for a column 0 <= z <= H drained at z = H (p = 0), no flow at z = 0."""
    p0 = terzaghi_p0(lam, mu, b, invM, load)
    c = terzaghi_c(lam, mu, b, invM, K, eta)
    zp = H - np.asarray(z, dtype=np.float64)
    out = np.zeros_like(zp)
    for m in range(terms):
        k = (2 * m + 1) * PI / (2 * H)
        out += 4.0 / ((2 * m + 1) * PI) * np.sin(k * zp) * np.exp(-k * k * c * t)
    return p0 * out
