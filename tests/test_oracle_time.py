"""Pins of the oracle's dG(r) time matrices (paper §Discretisation in Time)
against exact rationals, the characteristic polynomials of M_t^{-1} D and the
subdiagonal Pade stability functions (Radau IIA equivalence)."""
import os

import numpy as np
import pytest

from oracle import timebasis as tb

GOLD = os.path.join(os.path.dirname(__file__), "golden", "time_matrices_radau.txt")


def _golden():
    out = {}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        r, name, i, j, num, den = line.split()
        out[(int(r), name, i, j)] = float(num) / float(den)
    return out


def test_radau_matrices_match_exact_rationals():
    g = _golden()
    for (r, name, i, j), v in g.items():
        if name == "nodes":
            assert abs(tb.radau_right_nodes(r)[int(i)] - v) < 1e-14
            continue
        M, D = tb.radau_matrices(r)
        A = M if name == "Mt" else D
        assert abs(A[int(i), int(j)] - v) < 1e-13, (r, name, i, j)


def test_radau_mass_is_diagonal_with_radau_weights():
    # the (r+1)-point right-Radau rule is exact to degree 2r, so M_t is diagonal
    w2 = {0: [1.0], 1: [0.75, 0.25], 2: [(16 - np.sqrt(6)) / 36, (16 + np.sqrt(6)) / 36, 1.0 / 9.0]}
    for r in range(3):
        M, _ = tb.radau_matrices(r)
        assert np.allclose(M, np.diag(w2[r]), atol=1e-14)


@pytest.mark.parametrize("r,poly", [(0, [1, -1]), (1, [1, -4, 6]), (2, [1, -9, 36, -60])])
def test_eigenvalues_of_time_operator(r, poly):
    # eigenvalues of M_t^{-1} D are the reciprocals of the Pade poles' negatives:
    # z^2 - 4 z + 6 (r = 1: 2 +- i sqrt 2), z^3 - 9 z^2 + 36 z - 60 (r = 2)
    for basis in ("legendre", "radau"):
        M, D = tb.legendre_matrices(r) if basis == "legendre" else tb.radau_matrices(r)
        ev = np.sort_complex(np.linalg.eigvals(np.linalg.solve(M, D)))
        ref = np.sort_complex(np.roots(poly).astype(complex))
        assert np.allclose(ev, ref, atol=1e-10)


@pytest.mark.parametrize("r", [0, 1, 2])
def test_stability_function_is_subdiagonal_pade(r):
    for z in [0.01, 0.3, 1.0, 4.0, 25.0, 2.0 + 3.0j, 0.5 - 1.0j]:
        for basis in ("legendre", "radau"):
            got = tb.stability_function_dg(r, z, basis)
            ref = complex(tb.stability_function_closed_form(r, z))
            assert abs(got - ref) < 1e-12 * max(1.0, abs(ref))


def test_pade_approximates_exponential_to_order_2r_plus_1():
    for r in range(3):
        z1, z2 = 0.1, 0.05
        e1 = abs(tb.stability_function_closed_form(r, z1) - np.exp(-z1))
        e2 = abs(tb.stability_function_closed_form(r, z2) - np.exp(-z2))
        assert abs(np.log2(e1 / e2) - (2 * r + 2)) < 0.15  # local error O(z^{2r+2})


def test_basis_change_is_consistent():
    # a polynomial's Legendre and Radau coefficient vectors describe the same function
    for r in range(3):
        rng = np.random.default_rng(r)
        XL = rng.normal(size=r + 1)
        s = tb.radau_right_nodes(r)
        V = tb.legendre_vandermonde(s, r)
        XR = V @ XL
        t = np.linspace(0, 1, 7)
        assert np.allclose(tb.basis_values(t, r, "legendre").T @ XL, tb.basis_values(t, r, "radau").T @ XR)
