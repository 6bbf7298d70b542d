"""Differentiation workload: 3-D 32^3 hexes, dG(1), 16 slabs, layered log-normal
permeability; J = mean pressure over [0.4, 0.6]^3 at T^-.  The adjoint gradient
dJ/d(log K) (C ABI biot_adjoint_grad: transposed slab solves marched backwards with
end-state checkpoint recomputation) agrees with fourth-order central finite differences on
16 seeded unit-RMS directions, and checkpoint recomputation equals keeping every
forward slab."""
import numpy as np
import pytest

from gpu_common import C2, consolidation_bcs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_adjoint_gradient_matches_central_differences_32cube():
    from paper_1801_04984_gb300 import binding as B
    from paper_1801_04984_gb300.inputs import K0, fd_directions, layered_logk
    n, r, slabs, T = 32, 1, 16, 1.0
    g0 = layered_logk((n, n, n), layer_cells=4, std=1.5, seed=1801)
    ubc, fbc = consolidation_bcs(3)
    ctx = B.Context(3, (n, n, n), dict(C2, K=K0 * np.exp(g0)), r, ubc, fbc)
    f = torch.zeros(ctx.n_space, dtype=torch.float64, device="cuda")
    ctx.load_preset(B.LOAD_TRACTION_TOP, 1.0, f)
    j = torch.zeros_like(f)
    ctx.goal_mean_pressure([0.4] * 3, [0.6] * 3, j)
    U0 = torch.zeros_like(f)
    tol = 1e-12  # relative residual; the FP64 floor of this system lies near 1e-13
    dJ = torch.zeros(ctx.n_cells, dtype=torch.float64, device="cuda")
    J0 = ctx.adjoint_grad(T, slabs, [f], [[1, 0, 0, 0]], U0, j, dJ, tol=tol, mode=B.MIXED, recompute=True)
    dJ2 = torch.zeros_like(dJ)
    J1 = ctx.adjoint_grad(T, slabs, [f], [[1, 0, 0, 0]], U0, j, dJ2, tol=tol, mode=B.MIXED, recompute=False)
    assert J0 == J1 and torch.equal(dJ, dJ2)  # recomputation is bitwise equal to storing every slab
    grad = dJ.cpu().numpy()
    U = torch.zeros_like(f)

    def J(g):
        ctx.set_permeability(K0 * np.exp(g))
        ctx.march(T, slabs, [f], [[1, 0, 0, 0]], U0, U, tol=tol, mode=B.MIXED)
        return float(torch.dot(j, U).item())

    # fourth-order central differences: truncation O(eps^4) ~ 1e-11 of the derivative; every J
    # carries the solves' stopping noise (relative residual 1e-12: ~5e-13 absolute here), which
    # enters as ~1.5 noise / eps ~ 4e-10, i.e. ~4e-7 of the largest directional derivative
    # (~1e-3); second-order differences at eps 1e-4 sit at ~4e-6, the noise level itself
    eps = 2e-3
    fd, ad = [], []
    for d in fd_directions(ctx.n_cells, count=16, seed=4984):
        fd.append((8 * (J(g0 + eps * d) - J(g0 - eps * d)) - (J(g0 + 2 * eps * d) - J(g0 - 2 * eps * d))) / (12 * eps))
        ad.append(float(grad @ d))
    fd, ad = np.array(fd), np.array(ad)
    err = np.abs(fd - ad).max() / np.abs(ad).max()
    print("fourth-order FD vs adjoint: max error %.2e of the largest derivative" % err)
    assert err < 1e-6, (err, fd[:4], ad[:4])
