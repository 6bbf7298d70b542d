"""GPU slab operator (C ABI biot_apply_slab) against the oracle's assembled
slab matrix in the right-Radau basis: element-by-element, FP64 to 1e-12
relative, FP32 to its rounding level, forward and transposed, 2-D and 3-D,
r = 0, 1, 2, meshes spanning several tiles with ragged edges."""
import numpy as np
import pytest

from gpu_common import C2, consolidation_bcs, dirichlet_bcs, mixed_bcs
from oracle.slab import SlabProblem
from oracle.space import Mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ctx(n, r, bcs, K, co=C2, lo=None, hi=None):
    from paper_1801_04984_gb300 import binding as B
    ubc, fbc = bcs
    ctx = B.Context(len(n), n, dict(co, K=K), r, ubc, fbc, lo=lo, hi=hi)
    prob = SlabProblem(Mesh(n, lo=lo, hi=hi), dict(co, K=K), r, ubc, fbc)
    return ctx, prob


CASES = [
    ((9, 7), 1, "consolidation"), ((19, 3), 2, "mixed"), ((8, 8), 0, "dirichlet"),
    ((5, 3, 4), 1, "consolidation"), ((3, 9, 2), 2, "mixed"), ((4, 4, 4), 0, "dirichlet"),
]


@pytest.mark.parametrize("n,r,bc", CASES)
@pytest.mark.parametrize("transpose", [False, True])
def test_apply_fp64_matches_oracle(n, r, bc, transpose):
    d = len(n)
    bcs = {"consolidation": consolidation_bcs, "dirichlet": dirichlet_bcs, "mixed": mixed_bcs}[bc](d)
    rng = np.random.default_rng(hash((n, r, bc)) % 2**32)
    K = 1e-2 * np.exp(rng.normal(0, 1.5, size=int(np.prod(n))))
    hi = [1.0, 0.8, 1.3][:d]
    ctx, prob = _ctx(n, r, bcs, K, hi=hi)
    tau = 0.0625
    A = prob.operator(tau, "radau")
    if transpose:
        A = A.T.tocsr()
    x = rng.normal(size=prob.Nslab)
    y_ref = A @ x
    xd = torch.tensor(x, device="cuda")
    yd = torch.full_like(xd, np.nan)
    ctx.apply_slab(tau, xd, yd, transpose=transpose)
    y = yd.cpu().numpy()
    assert np.all(np.isfinite(y))
    rel = np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref)
    relmax = np.abs(y - y_ref).max() / np.abs(y_ref).max()
    assert rel < 1e-12 and relmax < 1e-12, (rel, relmax)


@pytest.mark.parametrize("n,r", [((9, 7), 1), ((5, 3, 4), 2)])
def test_apply_fp32_matches_oracle_to_rounding(n, r):
    d = len(n)
    rng = np.random.default_rng(5)
    K = 1e-2 * np.exp(rng.normal(0, 1.5, size=int(np.prod(n))))
    ctx, prob = _ctx(n, r, consolidation_bcs(d), K)
    tau = 0.0625
    x = rng.normal(size=prob.Nslab)
    y_ref = prob.operator(tau, "radau") @ x
    xd = torch.tensor(x, device="cuda", dtype=torch.float32)
    yd = torch.empty_like(xd)
    ctx.apply_slab(tau, xd, yd)
    rel = np.linalg.norm(yd.double().cpu().numpy() - y_ref) / np.linalg.norm(y_ref)
    assert rel < 2e-6, rel


def test_apply_is_deterministic():
    n, r = (5, 3, 4), 1
    rng = np.random.default_rng(9)
    K = 1e-2 * np.exp(rng.normal(0, 1.5, size=int(np.prod(n))))
    ctx, prob = _ctx(n, r, consolidation_bcs(3), K)
    xd = torch.tensor(rng.normal(size=prob.Nslab), device="cuda")
    y1, y2 = torch.empty_like(xd), torch.empty_like(xd)
    ctx.apply_slab(0.1, xd, y1)
    ctx.apply_slab(0.1, xd, y2)
    assert torch.equal(y1, y2)
