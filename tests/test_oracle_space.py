"""Pins of the oracle's spatial blocks (paper §Poroelasticity weak form,
§Discretisation in Space) against brute-force adaptive integration of
independently written basis functions, algebraic invariants (rigid motions,
patch test, exact divergence) and symmetry."""
import itertools

import numpy as np
import pytest
from numpy.polynomial import Polynomial
from scipy import integrate

from oracle.space import Mesh, SpatialBlocks, constraint_mask, U_DIRICHLET, U_ROLLER, U_NATURAL, F_NOFLOW, F_NATURAL

CO = dict(lam=1.7, mu=0.6, b=0.9, invM=0.1, eta=1.3)


def lagrange_1d(nodes):
    """Lagrange polynomials through `nodes` (physical coordinates)."""
    out = []
    for i, xi in enumerate(nodes):
        p = Polynomial([1.0])
        for j, xj in enumerate(nodes):
            if j != i:
                p = p * Polynomial([-xj, 1.0]) / (xi - xj)
        out.append(p)
    return out


def one_cell_bases(x0, y0, hx, hy):
    gs = [0.5 - np.sqrt(3) / 6, 0.5 + np.sqrt(3) / 6]
    Lx = lagrange_1d([x0, x0 + hx / 2, x0 + hx])
    Ly = lagrange_1d([y0, y0 + hy / 2, y0 + hy])
    Gx = lagrange_1d([x0 + hx * g for g in gs])
    Gy = lagrange_1d([y0 + hy * g for g in gs])
    # u: comp c, node (ax, ay), index c*9 + ax + 3 ay ; value = (phi, d/dx phi, d/dy phi)
    U = []
    for c in range(2):
        for ay in range(3):
            for ax in range(3):
                U.append((c, Lx[ax], Ly[ay]))
    Q = []
    for ay in range(2):  # comp 0: 3 along x, 2 Gauss across y ; index ax + 3 gy
        pass
    for gy in range(2):
        for ax in range(3):
            Q.append((0, Lx[ax], Gy[gy]))
    for ay in range(3):  # comp 1: index gx + 2 ay
        for gx in range(2):
            Q.append((1, Gx[gx], Ly[ay]))
    P = []
    for gy in range(2):
        for gx in range(2):
            P.append((Gx[gx], Gy[gy]))
    return U, Q, P


def _grad_u(f, x, y):
    c, px, py = f
    g = np.zeros((2, 2))
    g[c, 0] = px.deriv()(x) * py(y)
    g[c, 1] = px(x) * py.deriv()(y)
    return g


def _div_q(f, x, y):
    c, px, py = f
    return px.deriv()(x) * py(y) if c == 0 else px(x) * py.deriv()(y)


def _val_q(f, x, y):
    c, px, py = f
    v = np.zeros(2)
    v[c] = px(x) * py(y)
    return v


def _dbl(fun, x0, y0, hx, hy):
    val, _ = integrate.dblquad(lambda y, x: fun(x, y), x0, x0 + hx, y0, y0 + hy, epsabs=1e-13, epsrel=1e-13)
    return val


def test_one_cell_blocks_match_brute_force_integration():
    x0, y0, hx, hy = 0.0, 0.0, 0.5, 0.25
    m = Mesh((1, 1), lo=[x0, y0], hi=[x0 + hx, y0 + hy])
    K = 0.37
    blk = SpatialBlocks(m, dict(CO, K=np.array([K])))
    U, Q, P = one_cell_bases(x0, y0, hx, hy)
    lam, mu, eta = CO["lam"], CO["mu"], CO["eta"]
    A = blk.A.toarray()
    rng = np.random.default_rng(0)
    pairs = list(itertools.product(range(18), range(18)))
    for idx in rng.choice(len(pairs), 30, replace=False):
        i, j = pairs[idx]

        def a(x, y):
            gi, gj = _grad_u(U[i], x, y), _grad_u(U[j], x, y)
            ei, ej = 0.5 * (gi + gi.T), 0.5 * (gj + gj.T)
            return 2 * mu * np.sum(ei * ej) + lam * np.trace(gi) * np.trace(gj)
        assert abs(_dbl(a, x0, y0, hx, hy) - A[i, j]) < 1e-11, (i, j)
    E = blk.E.toarray()
    for i in range(0, 18, 3):
        for j in range(4):
            ref = _dbl(lambda x, y: np.trace(_grad_u(U[i], x, y)) * P[j][0](x) * P[j][1](y), x0, y0, hx, hy)
            assert abs(ref - E[i, j]) < 1e-12
    Mq = blk.Mq.toarray()
    Bd = blk.B.toarray()
    for i in range(12):
        for j in range(12):
            ref = eta / K * _dbl(lambda x, y: _val_q(Q[i], x, y) @ _val_q(Q[j], x, y), x0, y0, hx, hy)
            assert abs(ref - Mq[i, j]) < 1e-11
        for j in range(4):
            ref = _dbl(lambda x, y: _div_q(Q[i], x, y) * P[j][0](x) * P[j][1](y), x0, y0, hx, hy)
            assert abs(ref - Bd[j, i]) < 1e-12
    Mp = blk.Mp.toarray()
    for i in range(4):
        for j in range(4):
            ref = _dbl(lambda x, y: P[i][0](x) * P[i][1](y) * P[j][0](x) * P[j][1](y), x0, y0, hx, hy)
            assert abs(ref - Mp[i, j]) < 1e-13


def _node_coords(m):
    grids = np.meshgrid(*[m.lo[i] + m.h[i] / 2 * np.arange(m.u_shape[i]) for i in range(m.dim)], indexing="ij")
    return np.stack([g.transpose().reshape(-1) for g in grids], axis=1)  # x fastest


@pytest.mark.parametrize("n", [(3, 2), (2, 2, 3)])
def test_rigid_motions_in_kernel_and_symmetry(n):
    m = Mesh(n, hi=[1.0, 0.7, 1.3][: len(n)])
    blk = SpatialBlocks(m, dict(CO, K=np.linspace(0.1, 1.0, m.ncells)))
    X = _node_coords(m)
    d = m.dim
    motions = []
    for c in range(d):
        u = np.zeros((d, len(X)))
        u[c] = 1.0
        motions.append(u)
    for i, j in itertools.combinations(range(d), 2):
        u = np.zeros((d, len(X)))
        u[i] = -X[:, j]
        u[j] = X[:, i]
        motions.append(u)
    for u in motions:
        r = blk.A @ u.reshape(-1)
        assert np.abs(r).max() < 1e-12
        assert np.abs(blk.E.T @ u.reshape(-1)).max() < 1e-13  # rigid motions are divergence free
    for M in (blk.A, blk.Mq, blk.Mp):
        assert abs(M - M.T).max() < 1e-14
    Mp = blk.Mp.toarray()
    assert np.allclose(Mp, np.diag(np.diag(Mp)), atol=1e-15)
    assert abs(Mp.sum() - np.prod(m.hi - m.lo)) < 1e-13


def test_patch_test_linear_displacement():
    # linear u: constant stress, so every interior row of A u vanishes and
    # E^T u equals (div u) * int(psi)
    m = Mesh((3, 3, 2))
    blk = SpatialBlocks(m, dict(CO, K=np.ones(m.ncells)))
    X = _node_coords(m)
    G = np.array([[0.3, -1.1, 0.2], [0.5, 0.7, -0.4], [1.3, 0.1, 0.9]])
    u = (G @ X.T).reshape(-1)
    r = (blk.A @ u).reshape(3, -1)
    interior = np.all((X > 1e-12) & (X < 1 - 1e-12), axis=1)
    assert np.abs(r[:, interior]).max() < 1e-12
    assert np.allclose(blk.E.T @ u, np.trace(G) * blk.Mp.diagonal(), atol=1e-13)


def test_divergence_is_exact_and_flux_mass_scales_with_coefficient():
    m = Mesh((3, 2), hi=[1.5, 1.0])
    Kc = np.linspace(0.5, 2.0, m.ncells)
    blk = SpatialBlocks(m, dict(CO, K=Kc))
    # q = (x, 2y): RT1 interpolant is exact; div q = 3
    q = np.zeros(m.Nq)
    for c in range(2):
        shp = m.q_shapes[c]
        grids = np.meshgrid(*[np.arange(s) for s in shp], indexing="ij")
        co = [g.transpose().reshape(-1) for g in grids]
        along = co[c] * m.h[c] / 2
        q[m.off_q[c] - m.Nu: m.off_q[c] - m.Nu + m.Nq_c[c]] = (c + 1) * along
    assert np.allclose(blk.B @ q, 3.0 * blk.Mp.diagonal(), atol=1e-13)
    # constant q = (1, 0): q^T Mq q = sum_c eta/K_c |cell|
    q1 = np.zeros(m.Nq)
    q1[: m.Nq_c[0]] = 1.0
    assert abs(q1 @ (blk.Mq @ q1) - np.sum(CO["eta"] / Kc) * np.prod(m.h)) < 1e-12


def test_constraint_mask_counts():
    m = Mesh((2, 3, 4))
    mask = constraint_mask(m, [U_ROLLER] * 5 + [U_NATURAL], [F_NOFLOW] * 5 + [F_NATURAL])
    nx, ny, nz = m.u_shape
    # roller: u_x fixed on x faces, u_y on y faces, u_z on the bottom
    assert (mask[: m.nu_nodes] == 0).sum() == 2 * ny * nz
    assert (mask[m.nu_nodes: 2 * m.nu_nodes] == 0).sum() == 2 * nx * nz
    assert (mask[2 * m.nu_nodes: m.Nu] == 0).sum() == nx * ny
    assert (mask[m.off_q[2]: m.off_p] == 0).sum() == m.q_shapes[2][0] * m.q_shapes[2][1]
    assert np.all(mask[m.off_p:] == 1)
    mask = constraint_mask(m, [U_DIRICHLET] * 6, [F_NATURAL] * 6)
    assert (mask[: m.Nu] == 0).sum() == 3 * (m.nu_nodes - (nx - 2) * (ny - 2) * (nz - 2))
    assert np.all(mask[m.Nu:] == 1)
