"""dG(r) time-slab matrices (oracle; test infrastructure only).

Paper §Discretisation in Time: on each slab I_n = (t_{n-1}, t_n) the trial and
test functions are polynomials of degree r with values in the spatial space,
discontinuous across slab boundaries; testing with the discontinuous space gives
a time-marching scheme.  With s = (t - t_{n-1}) / tau in [0, 1] and basis
{phi_k}, the semi-discrete system S U' + A_s U = F becomes, per slab,

    sum_l [ D_kl S + tau (M_t)_kl A_s ] U_l = F_k + phi_k(0) S U(t_{n-1}^-)

    (M_t)_kl = int_0^1 phi_l phi_k ds,
    D_kl     = int_0^1 phi_l' phi_k ds + phi_l(0) phi_k(0)   (the jump term).

The oracle uses the shifted Legendre (modal) basis.  The nodal right-Radau
Lagrange basis used by the CUDA path is obtained by the exact change of basis
X_R = V X_L with V_im = P_m(s_i); tested equations transform with V^{-T}.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import Legendre, Polynomial


def legendre01(m: int) -> Polynomial:
    """Shifted Legendre polynomial P_m(2s - 1) as a power series in s."""
    return Legendre.basis(m, domain=[0.0, 1.0]).convert(kind=Polynomial, domain=[0.0, 1.0], window=[0.0, 1.0])


def _int01(p: Polynomial) -> float:
    ip = p.integ()
    return float(ip(1.0) - ip(0.0))


def legendre_matrices(r: int):
    """(M_t, D) in the shifted Legendre basis of degree <= r (exact polynomial integrals)."""
    P = [legendre01(m) for m in range(r + 1)]
    M = np.zeros((r + 1, r + 1))
    D = np.zeros((r + 1, r + 1))
    for k in range(r + 1):
        for l in range(r + 1):
            M[k, l] = _int01(P[l] * P[k])
            D[k, l] = _int01(P[l].deriv() * P[k]) + P[l](0.0) * P[k](0.0)
    return M, D


def radau_right_nodes(r: int) -> np.ndarray:
    """r+1 right-Radau points on [0, 1] (the last one is s = 1): roots of
    P_r(x) - P_{r+1}(x) on [-1, 1], mapped by s = (x + 1) / 2."""
    x = (Legendre.basis(r) - Legendre.basis(r + 1)).roots()
    x = np.sort(np.real(x))
    return (x + 1.0) / 2.0


def legendre_vandermonde(s: np.ndarray, r: int) -> np.ndarray:
    """V[i, m] = P_m(s_i)."""
    return np.array([[legendre01(m)(si) for m in range(r + 1)] for si in s])


def radau_matrices(r: int):
    """(M_t, D) in the Lagrange basis on the right-Radau nodes, by exact change of
    basis from the Legendre matrices: A_R = V^{-T} A_L V^{-1}."""
    ML, DL = legendre_matrices(r)
    V = legendre_vandermonde(radau_right_nodes(r), r)
    Vi = np.linalg.inv(V)
    return Vi.T @ ML @ Vi, Vi.T @ DL @ Vi


def basis_values(s: np.ndarray, r: int, basis: str) -> np.ndarray:
    """phi_k(s) for k = 0..r, shape (r+1, len(s)), in 'legendre' or 'radau' basis."""
    s = np.atleast_1d(np.asarray(s, dtype=np.float64))
    L = np.array([legendre01(m)(s) for m in range(r + 1)])
    if basis == "legendre":
        return L
    V = legendre_vandermonde(radau_right_nodes(r), r)
    # Radau Lagrange l_i = sum_m (V^{-1})_{m i} P_m
    return np.linalg.inv(V).T @ L


def stability_function_closed_form(r: int, z):
    """Subdiagonal Pade approximant of exp(-z) of type (r, r+1): the end-of-slab
    amplification of dG(r) for y' = -(z / tau) y."""
    z = np.asarray(z, dtype=np.complex128)
    if r == 0:
        return 1.0 / (1.0 + z)
    if r == 1:
        return (6.0 - 2.0 * z) / (6.0 + 4.0 * z + z * z)
    if r == 2:
        return 3.0 * (z * z - 8.0 * z + 20.0) / (z ** 3 + 9.0 * z * z + 36.0 * z + 60.0)
    raise ValueError("r <= 2")


def stability_function_dg(r: int, z: complex, basis: str = "legendre") -> complex:
    """End value after one slab of dG(r) applied to y' = -(z/tau) y, y(0^-) = 1:
    solve (D + z M_t) X = phi(0) and return sum_l X_l phi_l(1)."""
    M, D = legendre_matrices(r) if basis == "legendre" else radau_matrices(r)
    phi0 = basis_values(np.array([0.0]), r, basis)[:, 0]
    phi1 = basis_values(np.array([1.0]), r, basis)[:, 0]
    X = np.linalg.solve(D.astype(np.complex128) + z * M, phi0.astype(np.complex128))
    return complex(phi1 @ X)


def gauss01(npts: int):
    """Gauss-Legendre points and weights on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(npts)
    return (x + 1.0) / 2.0, w / 2.0
