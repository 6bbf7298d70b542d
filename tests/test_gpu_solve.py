"""GPU slab solves, marching and the adjoint (C ABI) against the oracle's
direct solves: FP64 to the solver tolerance, mixed precision to 1e-8 of the
FP64 result."""
import numpy as np
import pytest

from gpu_common import C1, C2, consolidation_bcs, dirichlet_bcs
from oracle.slab import SlabProblem, goal_vector_mean_p
from oracle.space import Mesh, load_vector
from oracle.exact import MMS2D

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup(n, r, bcs, K, co):
    from paper_1801_04984_gb300 import binding as B
    ubc, fbc = bcs
    return B.Context(len(n), n, dict(co, K=K), r, ubc, fbc), SlabProblem(Mesh(n), dict(co, K=K), r, ubc, fbc)


@pytest.mark.parametrize("n,r", [((8, 8), 1), ((16, 8), 2), ((4, 4, 4), 1), ((8, 4, 8), 0)])
def test_solve_fp64_matches_direct_solve(n, r):
    rng = np.random.default_rng(11)
    K = 1e-2 * np.exp(rng.normal(0, 1.5, size=int(np.prod(n))))
    ctx, prob = _setup(n, r, consolidation_bcs(len(n)), K, C2)
    tau = 1.0 / 16
    rhs = prob.mask * rng.normal(size=prob.Nslab)
    x_ref = prob.factor(tau, "radau").solve(rhs)
    x = torch.zeros(prob.Nslab, dtype=torch.float64, device="cuda")
    st = ctx.solve_slab(tau, torch.tensor(rhs, device="cuda"), x, tol=1e-10)
    xs = x.cpu().numpy()
    res = np.linalg.norm(rhs - prob.operator(tau, "radau") @ xs) / np.linalg.norm(rhs)
    assert res < 1e-10, (res, st)
    assert st["rel_residual"] < 1e-10


@pytest.mark.parametrize("n,r", [((8, 8), 1), ((4, 4, 4), 2)])
def test_mixed_precision_matches_fp64(n, r):
    rng = np.random.default_rng(12)
    K = 1e-2 * np.exp(rng.normal(0, 1.5, size=int(np.prod(n))))
    ctx, prob = _setup(n, r, consolidation_bcs(len(n)), K, C2)
    tau = 1.0 / 16
    rhs = torch.tensor(prob.mask * rng.normal(size=prob.Nslab), device="cuda")
    x64 = torch.zeros_like(rhs)
    x32 = torch.zeros_like(rhs)
    ctx.solve_slab(tau, rhs, x64, tol=1e-12)
    st = ctx.solve_slab(tau, rhs, x32, tol=1e-12, mode=2)
    rel = (torch.linalg.norm(x32 - x64) / torch.linalg.norm(x64)).item()
    assert rel < 1e-8, (rel, st)
    assert st["refinements"] >= 1


def test_march_mms_matches_oracle():
    # the 2-D manufactured-solution workload: 16 x 16 quads, dG(1), T = 1 in 8 slabs, FP64
    n, r = (16, 16), 1
    K = np.full(256, 1e-2)
    ctx, prob = _setup(n, r, dirichlet_bcs(2), K, C1)
    m = prob.mesh
    ex = MMS2D(1.0, 1.0, 0.9, 0.1, 1.0, 1e-2)
    load = lambda t: load_vector(m, t, f_u=ex.body_force, f_p=ex.source, p_bnd=ex.p_boundary,  # noqa: E731
                                 u_bc=prob.u_bc, f_bc=prob.f_bc)
    _, U_ref = prob.march(1.0, 8, load)
    from paper_1801_04984_gb300 import binding as B
    f0 = torch.zeros(ctx.n_space, dtype=torch.float64, device="cuda")
    f1 = torch.zeros_like(f0)
    ctx.load_preset(B.LOAD_MMS2D_CONST, 1.0, f0)
    ctx.load_preset(B.LOAD_MMS2D_LINEAR, 1.0, f1)
    # the presets equal the oracle's loads at t = 0 and their t-derivative
    assert np.allclose(f0.cpu().numpy() * prob.mask1, load(0.0) * prob.mask1, atol=1e-13)
    assert np.allclose(f1.cpu().numpy() * prob.mask1, (load(1.0) - load(0.0)) * prob.mask1, atol=1e-12)
    U = torch.zeros_like(f0)
    U0 = torch.zeros_like(f0)
    st = ctx.march(1.0, 8, [f0, f1], [[1, 0, 0, 0], [0, 1, 0, 0]], U0, U, tol=1e-12)
    rel = np.linalg.norm(U.cpu().numpy() - U_ref) / np.linalg.norm(U_ref)
    assert rel < 1e-9, (rel, st)


def test_adjoint_gradient_matches_oracle():
    n, r, slabs = (4, 4, 4), 1, 3
    from paper_1801_04984_gb300.inputs import layered_logk
    g0 = layered_logk(n, layer_cells=1, std=1.5, seed=3)
    K = 1e-2 * np.exp(g0)
    ctx, prob = _setup(n, r, consolidation_bcs(3), K, C2)
    from paper_1801_04984_gb300 import binding as B
    f = torch.zeros(ctx.n_space, dtype=torch.float64, device="cuda")
    ctx.load_preset(B.LOAD_TRACTION_TOP, 1.0, f)
    j = torch.zeros_like(f)
    ctx.goal_mean_pressure([0.4] * 3, [0.6] * 3, j)
    jo = goal_vector_mean_p(prob.mesh, np.array([0.4] * 3), np.array([0.6] * 3))
    assert np.abs(j.cpu().numpy() - jo).max() < 1e-13
    dJ = torch.zeros(ctx.n_cells, dtype=torch.float64, device="cuda")
    J = ctx.adjoint_grad(1.0, slabs, [f], [[1, 0, 0, 0]], None, j, dJ, tol=1e-13)
    load = lambda t: f.cpu().numpy()  # noqa: E731
    Xs, U = prob.march(1.0, slabs, load)
    assert abs(J - jo @ U) < 1e-10 * abs(jo @ U)
    Zs = prob.adjoint_march(1.0, slabs, Xs, jo)
    g_ref = prob.grad_logk(1.0, slabs, Xs, Zs)
    rel = np.linalg.norm(dJ.cpu().numpy() - g_ref) / np.linalg.norm(g_ref)
    assert rel < 1e-8, rel


def test_autograd_goal_gradient_is_the_adjoint_gradient():
    """torch.autograd through the goal functional returns the adjoint gradient, and J
    equals the goal weight applied to a forward march; a central difference along one
    seeded direction agrees to the solver tolerance."""
    from paper_1801_04984_gb300 import binding as B
    from paper_1801_04984_gb300.inputs import layered_logk
    n, r, slabs = (4, 4, 4), 1, 3
    g0 = layered_logk(n, layer_cells=1, std=1.5, seed=5)
    ubc, fbc = consolidation_bcs(3)
    ctx = B.Context(3, n, dict(C2, K=1e-2 * np.exp(g0)), r, ubc, fbc)
    f = torch.zeros(ctx.n_space, dtype=torch.float64, device="cuda")
    ctx.load_preset(B.LOAD_TRACTION_TOP, 1.0, f)
    j = torch.zeros_like(f)
    ctx.goal_mean_pressure([0.4] * 3, [0.6] * 3, j)
    U0 = torch.zeros_like(f)
    g = torch.tensor(g0, device="cuda", requires_grad=True)
    J = B.goal_of_logk(ctx, g, 1e-2, 1.0, slabs, [f], [[1, 0, 0, 0]], U0, j, tol=1e-13)
    J.backward()
    dJ = torch.zeros(ctx.n_cells, dtype=torch.float64, device="cuda")
    ctx.set_log_permeability(g0, 1e-2)  # the parametrisation the autograd path uses
    J_ref = ctx.adjoint_grad(1.0, slabs, [f], [[1, 0, 0, 0]], U0, j, dJ, tol=1e-13)
    assert J.item() == J_ref and torch.equal(g.grad, dJ)
    U = torch.zeros_like(f)
    ctx.march(1.0, slabs, [f], [[1, 0, 0, 0]], U0, U, tol=1e-13)
    assert abs(J_ref - torch.dot(j, U).item()) < 1e-10 * abs(J_ref)
    d = np.random.default_rng(7).normal(size=ctx.n_cells)
    eps = 1e-5
    Jp = B.goal_of_logk(ctx, torch.tensor(g0 + eps * d, device="cuda"), 1e-2, 1.0, slabs, [f], [[1, 0, 0, 0]], U0, j,
                        tol=1e-13).item()
    Jm = B.goal_of_logk(ctx, torch.tensor(g0 - eps * d, device="cuda"), 1e-2, 1.0, slabs, [f], [[1, 0, 0, 0]], U0, j,
                        tol=1e-13).item()
    fd = (Jp - Jm) / (2 * eps)
    ad = float(dJ.cpu().numpy() @ d)
    assert abs(fd - ad) < 1e-6 * abs(ad), (fd, ad)
    ctx.destroy()


@pytest.mark.parametrize("n,r", [((16, 16), 1), ((4, 4, 4), 1), ((32, 16), 0)])
def test_schur_multigrid_solves_match_direct_solve(n, r):
    """The flow block solved by one cell-centred multigrid V-cycle (opts schur_mg = 1):
    FP64 and mixed-precision slab solves still reach the direct solve's solution."""
    from paper_1801_04984_gb300 import binding as B
    rng = np.random.default_rng(21)
    K = 1e-2 * np.exp(rng.normal(0, 1.5, size=int(np.prod(n))))
    ubc, fbc = consolidation_bcs(len(n))
    ctx = B.Context(len(n), n, dict(C2, K=K), r, ubc, fbc, opts=dict(schur_mg=1))
    prob = SlabProblem(Mesh(n), dict(C2, K=K), r, ubc, fbc)
    tau = 1.0 / 8
    rhs = prob.mask * rng.normal(size=prob.Nslab)
    x_ref = prob.factor(tau, "radau").solve(rhs)
    for mode in (B.FP64, B.MIXED):
        x = torch.zeros(prob.Nslab, dtype=torch.float64, device="cuda")
        st = ctx.solve_slab(tau, torch.tensor(rhs, device="cuda"), x, tol=1e-11, mode=mode)
        rel = np.linalg.norm(x.cpu().numpy() - x_ref) / np.linalg.norm(x_ref)
        assert rel < 1e-8 and st["rel_residual"] < 1e-11, (mode, rel, st)
    ctx.destroy()


@pytest.mark.parametrize("n,r", [((6, 4), 0), ((4, 4, 4), 1)])
def test_dwr_time_estimate_matches_oracle(n, r):
    """Dual-weighted residual time-error indicators of the dG(r) march against dG(r+1)
    (C ABI biot_dwr_time_estimate) equal the oracle's slab by slab, and their sum equals
    the goal difference of two GPU marches (dG(r+1) minus dG(r))."""
    from paper_1801_04984_gb300 import binding as B
    from oracle.dwr import dwr_time_indicators
    rng = np.random.default_rng(50 + r)
    K = 1e-2 * np.exp(rng.normal(0, 1.0, size=int(np.prod(n))))
    d = len(n)
    ubc, fbc = consolidation_bcs(d)
    ctx = B.Context(d, n, dict(C2, K=K), r, ubc, fbc)
    ctx1 = B.Context(d, n, dict(C2, K=K), r + 1, ubc, fbc)
    f = torch.zeros(ctx.n_space, dtype=torch.float64, device="cuda")
    ctx.load_preset(B.LOAD_TRACTION_TOP, 1.0, f)
    j = torch.zeros_like(f)
    lo, hi = [0.25] * d, [0.75] * d
    ctx.goal_mean_pressure(lo, hi, j)
    U0 = torch.zeros_like(f)
    slabs = 5
    eta, eta_s, J = ctx.dwr_time_estimate(ctx1, 1.0, slabs, [f], [[1, 0, 0, 0]], U0, j, tol=1e-12)
    pr = SlabProblem(Mesh(n), dict(C2, K=K), r, ubc, fbc)
    pr1 = SlabProblem(Mesh(n), dict(C2, K=K), r + 1, ubc, fbc)
    F = f.cpu().numpy()
    jo = goal_vector_mean_p(pr.mesh, np.array(lo), np.array(hi))
    eta_o, J_o = dwr_time_indicators(pr, pr1, 1.0, slabs, lambda t: F, jo)
    assert abs(J - J_o) < 1e-10 * abs(J_o), (J, J_o)
    assert np.abs(np.array(eta_s) - eta_o).max() < 1e-9 * abs(J_o), (eta_s, eta_o)
    U1 = torch.zeros_like(f)
    ctx1.march(1.0, slabs, [f], [[1, 0, 0, 0]], U0, U1, tol=1e-12)
    diff = torch.dot(j, U1).item() - J
    assert abs(eta - diff) < 1e-9 * abs(J), (eta, diff)
    ctx.destroy()
    ctx1.destroy()


@pytest.mark.parametrize("n,r", [((8, 8), 0), ((4, 4, 4), 1)])
def test_fixed_stress_iterative_coupling_reaches_the_direct_solve(n, r):
    """The fixed-stress iterative coupling solve mode (flow with fixed mean stress, then
    deformation with fixed pressure, relaxed sweeps) converges to the direct solve's
    solution; it needs more sweeps than the monolithic FGMRES needs iterations."""
    from paper_1801_04984_gb300 import binding as B
    rng = np.random.default_rng(61 + r)
    K = 1e-2 * np.exp(rng.normal(0, 1.0, size=int(np.prod(n))))
    ctx, prob = _setup(n, r, consolidation_bcs(len(n)), K, C2)
    tau = 1.0 / 8
    rhs = prob.mask * rng.normal(size=prob.Nslab)
    x_ref = prob.factor(tau, "radau").solve(rhs)
    x = torch.zeros(prob.Nslab, dtype=torch.float64, device="cuda")
    st = ctx.solve_slab(tau, torch.tensor(rhs, device="cuda"), x, tol=1e-10, max_iters=5000, mode=B.FIXED_STRESS)
    rel = np.linalg.norm(x.cpu().numpy() - x_ref) / np.linalg.norm(x_ref)
    assert st["rel_residual"] < 1e-10 and rel < 1e-7, (rel, st)
    x2 = torch.zeros_like(x)
    st2 = ctx.solve_slab(tau, torch.tensor(rhs, device="cuda"), x2, tol=1e-10)
    assert st["iterations"] >= st2["iterations"], (st, st2)
    ctx.destroy()
