"""The FP32 displacement-row operator on meshes large enough for the z-marching kernel (65^3
nodes per component and more use it; smaller grids use the 8^3-tile kernel): ragged tiles in
every direction, every boundary code, all of its output stages.  The reference is the FP64
operator on the same (rounded) input, which the oracle pins element-wise (paper §Monolithic
Approach: the elasticity block A of A_s); the FP32 result must agree with it to FP32 rounding
on every entry, for the plain apply, the slab apply of r+1 temporal levels, and the multigrid
V-cycle whose smoothing steps and residuals run inside the kernel's output stage."""
import numpy as np
import pytest

from gpu_common import C2, consolidation_bcs, mixed_bcs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (cells, boundary codes): Q2 node grids 95 x 47 x 71 and 61 x 83 x 53 (> 1e5 nodes), ragged
# against the 28 x 8 output tiles and the z runs
CASES = [((47, 23, 35), "consolidation"), ((30, 41, 26), "mixed")]


def _ctx(n, bc, r=1):
    from paper_1801_04984_gb300 import binding as B
    bcs = consolidation_bcs(3) if bc == "consolidation" else mixed_bcs(3)
    K = 1e-2 * np.exp(np.random.default_rng(7).normal(0, 1.5, size=int(np.prod(n))))
    return B.Context(3, n, dict(C2, K=K), r, *bcs)


def _close(y32, y64, tol_max, tol_norm):
    y32 = y32.double()
    err = (y32 - y64).abs().max().item() / y64.abs().max().item()
    rel = (torch.linalg.norm(y32 - y64) / torch.linalg.norm(y64)).item()
    assert err < tol_max and rel < tol_norm, (err, rel)
    return err, rel


@pytest.mark.parametrize("n,bc", CASES)
def test_fp32_elasticity_matches_fp64_on_every_entry(n, bc):
    from paper_1801_04984_gb300 import binding as B
    ctx = _ctx(n, bc)
    g = torch.Generator(device="cuda").manual_seed(11)
    for smooth in (False, True):
        x32 = torch.rand(ctx.n_space, device="cuda", generator=g, dtype=torch.float32) * 2 - 1
        if smooth:  # a low-frequency field: A x is small against its terms (cancellation)
            i = torch.arange(ctx.n_space, device="cuda", dtype=torch.float32)
            x32 = torch.sin(i * 1e-4) + 0.01 * x32
        y32 = torch.full_like(x32, float("nan"))
        ctx.apply_part(B.PART_ELASTICITY, 0.05, x32, y32)
        y64 = torch.empty(ctx.n_space, dtype=torch.float64, device="cuda")
        ctx.apply_part(B.PART_ELASTICITY, 0.05, x32.double(), y64)
        _close(y32, y64, 1e-5, 2e-6 if not smooth else 2e-5)


@pytest.mark.parametrize("n,bc", CASES)
def test_fp32_slab_apply_matches_fp64(n, bc):
    ctx = _ctx(n, bc, r=2)
    x32 = torch.rand(ctx.n_slab, device="cuda", dtype=torch.float32, generator=torch.Generator(device="cuda").manual_seed(3)) - 0.5
    y32 = torch.full_like(x32, float("nan"))
    ctx.apply_slab(0.125, x32, y32)
    y64 = torch.empty(ctx.n_slab, dtype=torch.float64, device="cuda")
    ctx.apply_slab(0.125, x32.double(), y64)
    _close(y32, y64, 1e-5, 2e-6)


@pytest.mark.parametrize("n,bc", CASES)
def test_fp32_vcycle_matches_fp64(n, bc):
    """One V-cycle (Chebyshev-Jacobi smoothing and residuals fused into the operator's output
    stage, restriction, dense coarse solve, prolongation) is a fixed linear map: its FP32 and
    FP64 evaluations agree to FP32 rounding."""
    from paper_1801_04984_gb300 import binding as B
    ctx = _ctx(n, bc)
    x32 = torch.rand(ctx.n_space, device="cuda", dtype=torch.float32, generator=torch.Generator(device="cuda").manual_seed(5)) - 0.5
    y32 = torch.full_like(x32, float("nan"))
    ctx.apply_part(B.PART_VCYCLE, 0.05, x32, y32)
    y64 = torch.empty(ctx.n_space, dtype=torch.float64, device="cuda")
    ctx.apply_part(B.PART_VCYCLE, 0.05, x32.double(), y64)
    nu = 3 * int(np.prod([2 * m + 1 for m in n]))
    _close(y32[:nu], y64[:nu], 1e-4, 2e-5)
