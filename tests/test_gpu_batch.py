"""Batched instances (C ABI biot_setup_batch / biot_march_batch / biot_solve_batch).

A batched context holds several instances of one shape with their own
permeability fields; every kernel covers all of them in one launch.  Checked
here: the batched slab operator equals each instance's own operator (same
arithmetic per entry), the batched preconditioner equals the single-instance
one when the instances share a permeability field, batched marches match the
FP64 oracle's direct-solve marches instance by instance, and biot_solve_batch
over a ragged batch (several shapes, groups batched) equals solo marches."""
import numpy as np
import pytest

from gpu_common import C2, consolidation_bcs
from oracle.slab import SlabProblem
from oracle.space import Mesh, load_vector

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _perms(n, nb, seed):
    rng = np.random.default_rng(seed)
    return [1e-2 * np.exp(rng.normal(0, 1.5, size=int(np.prod(n)))) for _ in range(nb)]


def _interleave(xs, nt, N):
    """instance-major slab vectors -> one level-major batched vector"""
    return torch.cat([x[k * N:(k + 1) * N] for k in range(nt) for x in xs])


def _column(y, b, nb, nt, N):
    return torch.cat([y[(k * nb + b) * N:(k * nb + b + 1) * N] for k in range(nt)])


@pytest.mark.parametrize("n,r", [((8, 6), 1), ((4, 4, 4), 2), ((6, 4), 0)])
def test_batched_apply_equals_solo_applies(n, r):
    from paper_1801_04984_gb300 import binding as B
    nb = 3
    ubc, fbc = consolidation_bcs(len(n))
    Ks = _perms(n, nb, 5)
    ctxb = B.Context(len(n), n, dict(C2, K=np.concatenate(Ks)), r, ubc, fbc, nb=nb)
    solos = [B.Context(len(n), n, dict(C2, K=K), r, ubc, fbc) for K in Ks]
    N, nt = ctxb.n_space, ctxb.nt
    rng = np.random.default_rng(6)
    for dt in (torch.float64, torch.float32):
        for transpose in (False, True):
            xs = [torch.tensor(rng.normal(size=ctxb.n_slab), device="cuda", dtype=dt) for _ in range(nb)]
            yb = torch.empty(nb * ctxb.n_slab, device="cuda", dtype=dt)
            ctxb.apply_slab(0.1, _interleave(xs, nt, N), yb, transpose=transpose)
            for b in range(nb):
                ys = torch.empty_like(xs[b])
                solos[b].apply_slab(0.1, xs[b], ys, transpose=transpose)
                got = _column(yb, b, nb, nt, N)
                # same kernels, same per-entry arithmetic: identical up to FMA contraction choices
                err = (torch.linalg.norm(got - ys) / torch.linalg.norm(ys)).item()
                assert err < (1e-14 if dt == torch.float64 else 1e-6), (dt, transpose, b, err)
    for c in solos + [ctxb]:
        c.destroy()


@pytest.mark.parametrize("n,r", [((8, 8), 1), ((4, 4, 4), 2)])
def test_batched_preconditioner_equals_solo_for_shared_permeability(n, r):
    from paper_1801_04984_gb300 import binding as B
    nb = 3
    ubc, fbc = consolidation_bcs(len(n))
    K = _perms(n, 1, 7)[0]
    ctxb = B.Context(len(n), n, dict(C2, K=np.concatenate([K] * nb)), r, ubc, fbc, nb=nb)
    solo = B.Context(len(n), n, dict(C2, K=K), r, ubc, fbc)
    N, nt = ctxb.n_space, ctxb.nt
    rng = np.random.default_rng(8)
    for dt, tol in ((torch.float64, 1e-10), (torch.float32, 1e-4)):
        xs = [torch.tensor(rng.normal(size=ctxb.n_slab), device="cuda", dtype=dt) for _ in range(nb)]
        zb = torch.empty(nb * ctxb.n_slab, device="cuda", dtype=dt)
        ctxb.precondition(0.05, _interleave(xs, nt, N), zb)
        for b in range(nb):
            zs = torch.empty_like(xs[b])
            solo.precondition(0.05, xs[b], zs)
            got = _column(zb, b, nb, nt, N)
            err = (torch.linalg.norm(got - zs) / torch.linalg.norm(zs)).item()
            assert err < tol, (dt, b, err)
    ctxb.destroy()
    solo.destroy()


def _oracle_march(n, r, K, T, slabs):
    ubc, fbc = consolidation_bcs(len(n))
    prob = SlabProblem(Mesh(n), dict(C2, K=K), r, ubc, fbc)
    d = len(n)

    def trac(X, t, f):
        o = np.zeros((len(X), d))
        o[:, d - 1] = -1.0
        return o
    F = load_vector(prob.mesh, 0.0, traction=trac, u_bc=ubc, f_bc=fbc)
    _, U = prob.march(T, slabs, lambda t: F)
    return U


@pytest.mark.parametrize("n,r,nb", [((8, 8), 1, 4), ((4, 4, 4), 2, 2), ((8, 4), 0, 3)])
def test_batched_march_matches_oracle(n, r, nb):
    from paper_1801_04984_gb300 import binding as B
    ubc, fbc = consolidation_bcs(len(n))
    Ks = _perms(n, nb, 9)
    ctxb = B.Context(len(n), n, dict(C2, K=np.concatenate(Ks)), r, ubc, fbc, nb=nb)
    f = torch.zeros(ctxb.n_space, dtype=torch.float64, device="cuda")
    ctxb.load_preset(B.LOAD_TRACTION_TOP, 1.0, f)
    # instance b carries the load scaled by (b + 1): loads are per instance too
    terms = [[f * (b + 1)] for b in range(nb)]
    outs = [torch.zeros_like(f) for _ in range(nb)]
    rc, status, stats = ctxb.march_batch(0.5, 4, terms, [[1, 0, 0, 0]], None, outs, tol=1e-10)
    assert rc == 0 and all(s == 0 for s in status), (rc, status)
    for b in range(nb):
        U_ref = (b + 1) * _oracle_march(n, r, Ks[b], 0.5, 4)
        rel = np.linalg.norm(outs[b].cpu().numpy() - U_ref) / np.linalg.norm(U_ref)
        assert rel < 1e-8, (b, rel, stats[b])
        assert stats[b]["rel_residual"] < 1e-10 and stats[b]["iterations"] > 0, stats[b]
    ctxb.destroy()


def test_solve_batch_ragged_equals_solo_marches():
    from paper_1801_04984_gb300 import binding as B
    from paper_1801_04984_gb300.inputs import correlated_logk_2d
    ubc, fbc = consolidation_bcs(2)
    # shapes repeat, so groups of (8, 1) and (4, 2) run as batched contexts, the rest alone
    specs = [(4, 0), (8, 1), (4, 2), (8, 2), (8, 1), (16, 0), (8, 1), (4, 2)]
    inst = []
    for i, (n, r) in enumerate(specs):
        K = 1e-2 * np.exp(correlated_logk_2d(n, std=1.0, corr_cells=2.0, seed=100 + i))
        ns = 2 * (2 * n + 1) ** 2 + 2 * (2 * n + 1) * (2 * n) + (2 * n) ** 2
        inst.append(dict(dim=2, n=(n, n), coeffs=dict(C2, K=K), r=r, T=0.5, slabs=4, u_bc=ubc, f_bc=fbc,
                         load_kind=B.LOAD_TRACTION_TOP, load_value=1.0 + 0.25 * i, U_end=np.zeros(ns)))
    rc, status, stats = B.solve_batch(inst, tol=1e-10, mode=B.MIXED)
    assert rc == 0 and all(s == 0 for s in status), (rc, status)
    for i, (n, r) in enumerate(specs):
        K = inst[i]["coeffs"]["K"]
        ctx = B.Context(2, (n, n), dict(C2, K=K), r, ubc, fbc)
        f = torch.zeros(ctx.n_space, dtype=torch.float64, device="cuda")
        ctx.load_preset(B.LOAD_TRACTION_TOP, inst[i]["load_value"], f)
        U = torch.zeros_like(f)
        ctx.march(0.5, 4, [f], [[1, 0, 0, 0]], torch.zeros_like(f), U, tol=1e-10, mode=B.MIXED)
        ref = U.cpu().numpy()
        rel = np.linalg.norm(inst[i]["U_end"] - ref) / np.linalg.norm(ref)
        # two mixed-precision marches that each stop at relative residual 1e-10, at different
        # iterations (batched and solo reductions round differently), differ by up to the
        # conditioning times 1e-10: the bar is the mixed-precision error bar, 1e-8
        assert rel < 1e-8, (i, rel, stats[i])
        assert stats[i]["rel_residual"] < 1e-10
        ctx.destroy()
