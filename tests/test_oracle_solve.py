"""Pins of the oracle's slab system, direct solve, marching and adjoint
(paper §Monolithic Approach, §Discretisation in Time) against implicit Euler,
closed forms (manufactured solutions, Terzaghi), convergence orders, per-cell
mass balance and finite differences."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle.exact import MMS2D, PolyMMS2D, terzaghi_p0, terzaghi_pressure
from oracle.slab import SlabProblem, goal_vector_mean_p
from oracle.space import (F_NATURAL, F_NOFLOW, G2, U_DIRICHLET, U_NATURAL, U_ROLLER, Mesh, load_vector)
from oracle import timebasis as tb

C1 = dict(lam=1.0, mu=1.0, b=0.9, invM=0.1, eta=1.0)
C2 = dict(lam=1.0, mu=1.0, b=0.8, invM=0.05, eta=1.0)


def consolidation_bcs(d):
    ubc = [U_ROLLER] * (2 * d)
    ubc[-1] = U_NATURAL
    fbc = [F_NOFLOW] * (2 * d)
    fbc[-1] = F_NATURAL
    return ubc, fbc


def top_load(m, ubc, fbc, mag=1.0):
    d = m.dim

    def trac(X, t, f):
        out = np.zeros((len(X), d))
        out[:, -1] = -mag
        return out
    return lambda t: load_vector(m, t, traction=trac, u_bc=ubc, f_bc=fbc)


def field_errors(m, U, ex, t):
    cells, Lu, Lq, Lp = m.l2g()
    pts, W = m.quad(4)
    X = (m.lo + m.h * (cells[:, None, :] + pts[None, :, :])).reshape(-1, m.dim)
    Vu, _ = m.eval_u(pts)
    Vq, _ = m.eval_q(pts)
    Vp = m.eval_p(pts)
    Wf = np.tile(W, len(cells))
    uh = np.einsum("jqa,cj->cqa", Vu, U[Lu]).reshape(-1, m.dim)
    qh = np.einsum("jqa,cj->cqa", Vq, U[Lq]).reshape(-1, m.dim)
    ph = np.einsum("jq,cj->cq", Vp, U[Lp]).reshape(-1)
    return (np.sqrt(np.sum(Wf[:, None] * (uh - ex.u(X, t)) ** 2)),
            np.sqrt(np.sum(Wf[:, None] * (qh - ex.q(X, t)) ** 2)),
            np.sqrt(np.sum(Wf * (ph - ex.p(X, t)) ** 2)))


def mms_problem(n, r, ex_cls=MMS2D):
    m = Mesh((n, n))
    co = dict(C1, K=np.full(m.ncells, 1e-2))
    ex = ex_cls(1.0, 1.0, 0.9, 0.1, 1.0, 1e-2)
    prob = SlabProblem(m, co, r, [U_DIRICHLET] * 4, [F_NATURAL] * 4)
    load = lambda t: load_vector(m, t, f_u=ex.body_force, f_p=ex.source, p_bnd=ex.p_boundary,  # noqa: E731
                                 u_bc=prob.u_bc, f_bc=prob.f_bc)
    return m, prob, ex, load


def test_dg0_is_implicit_euler_with_averaged_load():
    m, prob, ex, load = mms_problem(4, 0)
    Xs, U = prob.march(1.0, 5, load)
    # implicit Euler written from the semi-discrete form: (S + tau A_s) U_n = S U_{n-1} + int F
    blk = prob.blocks
    A_s, S, mask = blk.stationary(), blk.storage(), prob.mask1
    tau = 0.2
    Md = sp.diags(mask)
    L = (Md @ (S + tau * A_s) @ Md + sp.diags(1 - mask)).tocsc()
    Ue = np.zeros(m.N)
    xg, wg = np.polynomial.legendre.leggauss(10)
    for n in range(5):
        Fint = sum(0.5 * tau * w * load(n * tau + tau * (x + 1) / 2) for x, w in zip(xg, wg))
        Ue = spla.spsolve(L, mask * (S @ Ue + Fint))
        assert np.abs(Xs[n] - Ue).max() < 1e-12 * max(1.0, np.abs(Ue).max())


def test_mms_space_orders():
    errs = []
    for n in (4, 8, 16):
        m, prob, ex, load = mms_problem(n, 1)
        _, U = prob.march(1.0, 8, load)
        errs.append(field_errors(m, U, ex, 1.0))
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert np.all(rates[:, 0] > 2.9)   # u in L2: O(h^3)
    assert np.all(rates[:, 1] > 1.9)   # q in L2: O(h^2)
    assert np.all(rates[:, 2] > 1.9)   # p in L2: O(h^2)


@pytest.mark.parametrize("r", [0, 1, 2])
def test_time_order_at_slab_ends(r):
    # constant load from a (near-)undrained start: the nodal error is O(tau^{2r+1})
    m = Mesh((1, 8))
    co = dict(C2, K=np.full(m.ncells, 1e-2))
    ubc, fbc = consolidation_bcs(2)
    load = top_load(m, ubc, fbc)
    _, U0 = SlabProblem(m, co, 0, ubc, fbc).march(1e-8, 1, load)
    prob = SlabProblem(m, co, r, ubc, fbc)
    _, Uref = prob.march(1.0 + 1e-8, 1024, load, U0=U0, t_start=1e-8)
    Ns = [4, 8, 16]
    errs = np.array([np.abs(prob.march(1.0 + 1e-8, N, load, U0=U0, t_start=1e-8)[1] - Uref).max() for N in Ns])
    rates = np.log2(errs[:-1] / errs[1:])
    assert rates[-1] > 2 * r + 1 - 0.15, rates


@pytest.mark.parametrize("r", [0, 1, 2])
def test_time_order_with_time_dependent_forcing(r):
    # forcing that varies in time enters the algebraic (quasi-static u and Darcy)
    # rows through its L2 projection on each slab: O(tau^{r+1}) at slab ends
    m, prob, ex, load = mms_problem(2, r, PolyMMS2D)
    cells, Lu, Lq, Lp = m.l2g()
    pts = np.array([[G2[a[0]], G2[a[1]]] for a in m.local_p()])
    Xp = ((cells[:, None, :] + pts[None, :, :]) * m.h).reshape(-1, 2)
    pe = ex.p(Xp, 1.0)
    errs = np.array([np.abs(prob.march(1.0, N, load)[1][Lp].reshape(-1) - pe).max() for N in (32, 64, 128)])
    rates = np.log2(errs[:-1] / errs[1:])
    assert abs(rates[-1] - (r + 1)) < 0.1, rates


@pytest.mark.parametrize("dim,n", [(2, (2, 32)), (3, (2, 2, 16))])
def test_terzaghi_closed_form(dim, n):
    m = Mesh(n)
    co = dict(C2, K=np.full(m.ncells, 1e-2))
    ubc, fbc = consolidation_bcs(dim)
    prob = SlabProblem(m, co, 1, ubc, fbc)
    _, U = prob.march(1.0, 16, top_load(m, ubc, fbc))
    pg = U[m.off_p:].reshape(m.p_shape[::-1]).reshape(m.p_shape[-1], -1)
    iz = np.arange(m.p_shape[-1])
    zc = (iz // 2 + G2[iz % 2]) * m.h[-1]
    ex = terzaghi_pressure(zc, 1.0, 1.0, 1.0, 0.8, 0.05, 1e-2, 1.0)
    p0 = terzaghi_p0(1.0, 1.0, 0.8, 0.05)
    assert abs(p0 - 1.0127) < 1e-4
    assert np.abs(pg - ex[:, None]).max() / p0 < 1e-4
    assert np.ptp(pg, axis=1).max() < 1e-12  # the solution is one-dimensional


def test_per_cell_mass_balance():
    # b (div u_t, w) + (1/M)(p_t, w) + (div q, w) - (f, w), tested slab-wise with
    # psi_g phi_k (plus the jump), evaluated by quadrature of the solution fields
    m, prob, ex, load = mms_problem(4, 1)
    Xs, _ = prob.march(1.0, 4, load)
    r, tau, N = 1, 0.25, m.N
    cells, Lu, Lq, Lp = m.l2g()
    pts, W = m.quad(4)  # the load's own spatial rule (exact for the polynomial terms)
    _, Gu = m.eval_u(pts)
    _, Dq = m.eval_q(pts)
    Vp = m.eval_p(pts)
    divu = np.trace(Gu, axis1=2, axis2=3)
    st, wt = tb.gauss01(8)  # the load's own time rule
    phi = tb.basis_values(st, r, "legendre")
    dphi = np.array([tb.legendre01(k).deriv()(st) for k in range(r + 1)])
    phi0 = tb.basis_values(np.array([0.0]), r, "legendre")[:, 0]
    X3 = (m.lo + m.h * (cells[:, None, :] + pts[None, :, :])).reshape(-1, 2)
    Uprev = np.zeros(N)
    worst = 0.0
    for n, X in enumerate(Xs):
        Xk = X.reshape(r + 1, N)
        bal = np.zeros((len(cells), 4, r + 1))
        for q_t in range(len(st)):
            t = n * tau + tau * st[q_t]
            U_t = dphi[:, q_t] @ Xk / tau
            U_v = phi[:, q_t] @ Xk
            du = np.einsum("jq,cj->cq", divu, U_t[Lu])
            dp = np.einsum("jq,cj->cq", Vp, U_t[Lp])
            dq = np.einsum("jq,cj->cq", Dq, U_v[Lq])
            f = ex.source(X3, t).reshape(len(cells), -1)
            integrand = 0.9 * du + 0.1 * dp + dq - f
            cellint = np.einsum("cq,gq,q->cg", integrand, Vp, W)
            bal += tau * wt[q_t] * cellint[:, :, None] * phi[None, None, :, q_t]
        jump = Xk.T @ phi0 - Uprev
        dj = np.einsum("jq,cj->cq", divu, jump[Lu]) * 0.9 + 0.1 * np.einsum("jq,cj->cq", Vp, jump[Lp])
        bal += np.einsum("cq,gq,q->cg", dj, Vp, W)[:, :, None] * phi0[None, None, :]
        worst = max(worst, np.abs(bal).max())
        Uprev = prob.end_value(X)
    assert worst < 1e-12


def test_layered_3d_reduces_to_2d():
    g = np.array([0.3, -1.2, 2.0, 0.1])
    K1 = 1e-2 * np.exp(np.repeat(g, 4))  # 4-cell layers along the vertical axis
    m3 = Mesh((2, 2, 16))
    m2 = Mesh((2, 16))
    K3 = np.repeat(K1, 4)
    K2 = np.repeat(K1, 2)
    out = []
    for m, K in ((m3, K3), (m2, K2)):
        ubc, fbc = consolidation_bcs(m.dim)
        prob = SlabProblem(m, dict(C2, K=K), 1, ubc, fbc)
        _, U = prob.march(1.0, 8, top_load(m, ubc, fbc))
        pg = U[m.off_p:].reshape(m.p_shape[::-1]).reshape(m.p_shape[-1], -1)
        out.append(pg[:, 0])
    assert np.abs(out[0] - out[1]).max() < 1e-12


def test_legendre_and_radau_solves_agree():
    m, prob, ex, load = mms_problem(4, 2)
    _, UL = prob.march(1.0, 3, load, basis="legendre")
    XsR, UR = prob.march(1.0, 3, load, basis="radau")
    assert np.abs(UL - UR).max() < 1e-12
    # Radau basis: the last temporal DoF is the end value
    assert np.abs(XsR[-1].reshape(3, -1)[-1] - UR).max() < 1e-14


def test_goal_functional_is_exact_mean():
    m = Mesh((5, 5, 5))
    j = goal_vector_mean_p(m, np.array([0.4] * 3), np.array([0.6] * 3))
    U = np.zeros(m.N)
    # p(x) = 1 + 2x - y + 3z at Gauss points (exact in DGQ1); mean over the box = 1 + 1 - .5 + 1.5
    grids = np.meshgrid(*[np.arange(s) for s in m.p_shape], indexing="ij")
    co = [gg.transpose().reshape(-1) for gg in grids]
    xyz = [(co[i] // 2 + G2[co[i] % 2]) * m.h[i] for i in range(3)]
    U[m.off_p:] = 1 + 2 * xyz[0] - xyz[1] + 3 * xyz[2]
    assert abs(j @ U - 3.0) < 1e-13


def test_adjoint_gradient_matches_finite_differences():
    from paper_1801_04984_gb300.inputs import layered_logk, fd_directions
    m = Mesh((2, 2, 4))
    g0 = layered_logk(m.n, layer_cells=1, std=1.5, seed=7)
    ubc, fbc = consolidation_bcs(3)
    load = top_load(m, ubc, fbc)
    jv = goal_vector_mean_p(m, np.array([0.4] * 3), np.array([0.6] * 3))

    def J(g):
        prob = SlabProblem(m, dict(C2, K=1e-2 * np.exp(g)), 1, ubc, fbc)
        Xs, U = prob.march(1.0, 3, load)
        return jv @ U, prob, Xs
    J0, prob, Xs = J(g0)
    Zs = prob.adjoint_march(1.0, 3, Xs, jv)
    grad = prob.grad_logk(1.0, 3, Xs, Zs)
    for d in fd_directions(m.ncells, count=3, seed=4984):
        eps = 1e-5
        fd = (J(g0 + eps * d)[0] - J(g0 - eps * d)[0]) / (2 * eps)
        assert abs(fd - grad @ d) < 1e-8 * max(1.0, abs(fd)), (fd, grad @ d)


@pytest.mark.parametrize("n,r", [((3, 2), 1), ((2, 3, 2), 2)])
def test_rowwise_apply_matches_assembled_operator(n, r):
    from oracle.slab import CellwiseSlab, apply_rows
    m = Mesh(n)
    ubc, fbc = consolidation_bcs(m.dim)
    prob = SlabProblem(m, dict(C2, K=np.linspace(0.01, 0.1, m.ncells)), r, ubc, fbc)
    X = np.random.default_rng(3).normal(size=prob.Nslab)
    y = prob.operator(0.3, "radau") @ X
    rows = np.arange(prob.Nslab)
    assert np.abs(apply_rows(prob, 0.3, X, rows) - y).max() < 1e-13 * np.abs(y).max()
    # the assembly-free form used for full-size parity gives the same rows
    light = CellwiseSlab(m, dict(C2, K=np.linspace(0.01, 0.1, m.ncells)), r, ubc, fbc)
    assert np.abs(apply_rows(light, 0.3, X, rows) - y).max() < 1e-13 * np.abs(y).max()


@pytest.mark.parametrize("r", [0, 1])
def test_dwr_time_indicators_sum_to_the_goal_difference(r):
    """Dual-weighted residual of the dG(r) solution in the dG(r+1) system: the slab
    indicators sum to J(U_{r+1}) - J(U_r), computed independently by two direct-solve
    marches (an identity of the block-bidiagonal slab system), and they are not all of
    one size: the first slabs, where the sudden load acts, carry most of the error."""
    from oracle.dwr import dwr_time_indicators
    n = (6, 4)
    rng = np.random.default_rng(40 + r)
    co = dict(C2, K=1e-2 * np.exp(rng.normal(0, 1.0, size=24)))
    ubc, fbc = consolidation_bcs(2)
    m = Mesh(n)
    pr = SlabProblem(m, co, r, ubc, fbc)
    pr1 = SlabProblem(m, co, r + 1, ubc, fbc)

    def trac(X, t, f):
        o = np.zeros((len(X), 2))
        o[:, 1] = -1.0
        return o
    F = load_vector(m, 0.0, traction=trac, u_bc=ubc, f_bc=fbc)
    j = goal_vector_mean_p(m, np.array([0.25, 0.25]), np.array([0.75, 0.75]))
    eta, J_r = dwr_time_indicators(pr, pr1, 1.0, 5, lambda t: F, j)
    _, U1 = pr1.march(1.0, 5, lambda t: F)
    _, U0 = pr.march(1.0, 5, lambda t: F)
    assert abs(J_r - j @ U0) < 1e-14 * abs(J_r)
    diff = j @ U1 - j @ U0
    # identity up to the rounding of the two goal values it is the difference of
    assert abs(eta.sum() - diff) < 1e-12 * abs(J_r), (eta.sum(), diff, J_r)
    assert abs(eta[0]) > abs(eta[-1])
