"""Failure handling and restart on the GPU path, with every failure made on the host:

* a non-finite right-hand side gives BIOT_EINVAL before any iteration;
* an iteration budget too small for the tolerance gives BIOT_ENOCONV with a finite best
  iterate whose residual is reported;
* a march stopped after slab k (the host simply stops calling) and resumed from the
  returned state U(t_k^-) reproduces the uninterrupted march bitwise (paper
  §Discretisation in Time: U(t_n^-) is all a slab passes on), also with loads that
  depend on time, and also on a freshly created context."""
import numpy as np
import pytest

from gpu_common import C2, consolidation_bcs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ctx(n=(4, 3, 5), r=1, seed=3):
    from paper_1801_04984_gb300 import binding as B
    K = 1e-2 * np.exp(np.random.default_rng(seed).normal(0, 1.0, size=int(np.prod(n))))
    return B.Context(len(n), n, dict(C2, K=K), r, *consolidation_bcs(len(n)))


def test_non_finite_rhs_is_rejected():
    from paper_1801_04984_gb300 import binding as B
    ctx = _ctx()
    rhs = torch.ones(ctx.n_slab, dtype=torch.float64, device="cuda")
    rhs[17] = float("nan")
    x = torch.zeros_like(rhs)
    for mode in (B.FP64, B.MIXED):
        with pytest.raises(B.BiotError) as e:
            ctx.solve_slab(0.1, rhs, x, mode=mode)
        assert e.value.code == B.EINVAL


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_iteration_budget_gives_noconv_with_finite_best_iterate(mode):
    from paper_1801_04984_gb300 import binding as B
    ctx = _ctx()
    rng = np.random.default_rng(5)
    rhs = torch.tensor(rng.normal(size=ctx.n_slab), device="cuda")
    x = torch.zeros_like(rhs)
    st = ctx.solve_slab(0.1, rhs, x, tol=1e-14, max_iters=3, mode=B.FP64 if mode == "fp64" else B.MIXED,
                        allow_noconv=True)
    assert st["iterations"] <= 3 + 30  # MIXED: the budget bounds the inner iterations of the cycles it starts
    assert np.isfinite(st["rel_residual"]) and 1e-14 < st["rel_residual"] < 1.0
    assert torch.isfinite(x).all() and torch.linalg.norm(x) > 0
    with pytest.raises(B.BiotError) as e:
        ctx.solve_slab(0.1, rhs, torch.zeros_like(rhs), tol=1e-14, max_iters=3,
                       mode=B.FP64 if mode == "fp64" else B.MIXED)
    assert e.value.code == B.ENOCONV


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_stopped_and_resumed_march_is_bitwise_the_uninterrupted_march(mode):
    from paper_1801_04984_gb300 import binding as B
    m = B.FP64 if mode == "fp64" else B.MIXED
    ctx = _ctx()
    f = torch.zeros(ctx.n_space, dtype=torch.float64, device="cuda")
    ctx.load_preset(B.LOAD_TRACTION_TOP, 1.0, f)
    tcoef = [[0.5, 1.0, -0.3, 0.0]]  # load magnitude varying in time
    T, slabs, k = 1.0, 6, 2
    U0 = torch.zeros_like(f)
    U_full = torch.zeros_like(f)
    X_full = torch.empty(slabs * ctx.n_slab, dtype=torch.float64, device="cuda")
    ctx.march(T, slabs, [f], tcoef, U0, U_full, X_all=X_full, mode=m)
    for fresh in (False, True):
        c = _ctx() if fresh else ctx
        U_k = torch.zeros_like(f)
        X_a = torch.empty(k * ctx.n_slab, dtype=torch.float64, device="cuda")
        c.march_resume(T, slabs, 0, k, [f], tcoef, U0, U_k, X_all=X_a, mode=m)
        if fresh:  # the restart runs in a new context (as after the host process stopped)
            c = _ctx()
        U_end = torch.zeros_like(f)
        X_b = torch.empty((slabs - k) * ctx.n_slab, dtype=torch.float64, device="cuda")
        c.march_resume(T, slabs, k, slabs - k, [f], tcoef, U_k.cpu().numpy(), U_end, X_all=X_b, mode=m)
        assert torch.equal(X_a, X_full[:k * ctx.n_slab]), fresh
        assert torch.equal(X_b, X_full[k * ctx.n_slab:]), fresh
        assert torch.equal(U_end, U_full), fresh
    with pytest.raises(B.BiotError) as e:
        ctx.march_resume(T, slabs, 5, 2, [f], tcoef, U0, torch.zeros_like(f))
    assert e.value.code == B.EINVAL
