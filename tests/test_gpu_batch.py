"""Batched marches (C ABI biot_solve_batch): every instance of a ragged batch
(mesh size, time order r, permeability field) equals its own solo march."""
import numpy as np
import pytest

from gpu_common import C2, consolidation_bcs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_batch_instances_equal_solo_marches():
    from paper_1801_04984_gb300 import binding as B
    from paper_1801_04984_gb300.inputs import correlated_logk_2d
    ubc, fbc = consolidation_bcs(2)
    specs = [(4, 0), (8, 1), (4, 2), (8, 2), (8, 1), (16, 0)]
    inst = []
    for i, (n, r) in enumerate(specs):
        K = 1e-2 * np.exp(correlated_logk_2d(n, std=1.0, corr_cells=2.0, seed=100 + i))
        ctx = B.Context(2, (n, n), dict(C2, K=K), r, ubc, fbc)
        inst.append(dict(dim=2, n=(n, n), coeffs=dict(C2, K=K), r=r, T=0.5, slabs=4, u_bc=ubc, f_bc=fbc,
                         load_kind=B.LOAD_TRACTION_TOP, load_value=1.0, U_end=np.zeros(ctx.n_space)))
        ctx.destroy()
    rc, status, stats = B.solve_batch(inst, workers=3, tol=1e-10, mode=B.MIXED)
    assert rc == 0 and all(s == 0 for s in status), (rc, status)
    for i, (n, r) in enumerate(specs):
        K = inst[i]["coeffs"]["K"]
        ctx = B.Context(2, (n, n), dict(C2, K=K), r, ubc, fbc)
        f = torch.zeros(ctx.n_space, dtype=torch.float64, device="cuda")
        ctx.load_preset(B.LOAD_TRACTION_TOP, 1.0, f)
        U = torch.zeros_like(f)
        ctx.march(0.5, 4, [f], [[1, 0, 0, 0]], torch.zeros_like(f), U, tol=1e-10, mode=B.MIXED)
        ref = U.cpu().numpy()
        rel = np.linalg.norm(inst[i]["U_end"] - ref) / np.linalg.norm(ref)
        assert rel < 1e-9, (i, rel, stats[i])
        assert stats[i]["rel_residual"] < 1e-10
        ctx.destroy()
