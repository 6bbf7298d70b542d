"""The hand-derived manufactured loads (oracle.exact) re-derived symbolically
from the strong form of the paper's §Poroelasticity system."""
import numpy as np
import pytest

from oracle.exact import MMS2D, PolyMMS2D


def _symbolic_loads(u_expr, p_expr, lam, mu, b, invM, eta, K):
    sympy = pytest.importorskip("sympy")
    x, y, t = sympy.symbols("x y t")
    u = [u_expr[0](x, y, t), u_expr[1](x, y, t)]
    p = p_expr(x, y, t)
    X = [x, y]
    eps = [[(sympy.diff(u[i], X[j]) + sympy.diff(u[j], X[i])) / 2 for j in range(2)] for i in range(2)]
    divu = sympy.diff(u[0], x) + sympy.diff(u[1], y)
    sig = [[2 * mu * eps[i][j] + (lam * divu - b * p) * (1 if i == j else 0) for j in range(2)] for i in range(2)]
    fu = [-(sympy.diff(sig[i][0], x) + sympy.diff(sig[i][1], y)) for i in range(2)]
    q = [-(K / eta) * sympy.diff(p, X[i]) for i in range(2)]
    f = b * sympy.diff(divu, t) + invM * sympy.diff(p, t) + sympy.diff(q[0], x) + sympy.diff(q[1], y)
    return [sympy.lambdify((x, y, t), e, "numpy") for e in fu + [f]]


@pytest.mark.parametrize("cls", [MMS2D, PolyMMS2D])
def test_manufactured_loads_match_symbolic_derivation(cls):
    sympy = pytest.importorskip("sympy")
    lam, mu, b, invM, eta, K = 1.3, 0.7, 0.9, 0.1, 1.1, 1e-2
    ex = cls(lam, mu, b, invM, eta, K)
    if cls is MMS2D:
        ue = (lambda x, y, t: sympy.sin(sympy.pi * x) * sympy.sin(sympy.pi * y) * t,) * 2
        pe = lambda x, y, t: sympy.cos(sympy.pi * x) * sympy.cos(sympy.pi * y) * t  # noqa: E731
    else:
        g = lambda t: sympy.sin(3 * t) + 1 - sympy.cos(3 * t)  # noqa: E731
        ue = (lambda x, y, t: x * (1 - x) * y * (1 - y) * g(t), lambda x, y, t: 0 * x)
        pe = lambda x, y, t: (x + 2 * y) * g(t)  # noqa: E731
    fx, fy, f = _symbolic_loads(ue, pe, lam, mu, b, invM, eta, K)
    rng = np.random.default_rng(1)
    X = rng.uniform(0, 1, size=(50, 2))
    for t in (0.0, 0.37, 1.0):
        bf = ex.body_force(X, t)
        assert np.allclose(bf[:, 0], fx(X[:, 0], X[:, 1], t) + 0 * X[:, 0], atol=1e-12)
        assert np.allclose(bf[:, 1], fy(X[:, 0], X[:, 1], t) + 0 * X[:, 0], atol=1e-12)
        assert np.allclose(ex.source(X, t), f(X[:, 0], X[:, 1], t) + 0 * X[:, 0], atol=1e-12)
