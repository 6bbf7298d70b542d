"""Preconditioner components (C ABI biot_apply_part) against the oracle's
assembled blocks: exact inverse of the Darcy mass by lines, the flux-pressure
Schur complement of the dG(0)-type diagonal block (paper §Monolithic Approach,
L_j with the fixed-stress term), the elasticity block, and the contraction of
the multigrid V-cycle."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from gpu_common import C2, consolidation_bcs, mixed_bcs
from oracle.space import Mesh, SpatialBlocks, constraint_mask

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [((9, 7), consolidation_bcs(2)), ((6, 5, 4), consolidation_bcs(3)), ((5, 4, 6), mixed_bcs(3))]


def _ctx(n, bcs, K, exact=0):
    from paper_1801_04984_gb300 import binding as B
    ubc, fbc = bcs
    return B.Context(len(n), n, dict(C2, K=K), 1, ubc, fbc, opts=dict(flux_mass_exact=exact))


@pytest.mark.parametrize("n,bcs", CASES)
def test_flux_mass_inverse_and_schur(n, bcs):
    from paper_1801_04984_gb300 import binding as B
    rng = np.random.default_rng(21)
    K = 1e-2 * np.exp(rng.normal(0, 1.5, size=int(np.prod(n))))
    ctx = _ctx(n, bcs, K, exact=1)
    m = Mesh(n)
    blk = SpatialBlocks(m, dict(C2, K=K))
    mask = constraint_mask(m, *bcs)
    fq = mask[m.Nu:m.off_p] == 1.0
    tau = 0.07
    x = rng.normal(size=m.N)
    xd = torch.tensor(x, device="cuda")
    yd = torch.empty_like(xd)
    ctx.apply_part(B.PART_FLUX_MASS_INV, tau, xd, yd)
    y = yd.cpu().numpy()
    Mq = blk.Mq.tocsr()[fq][:, fq]
    xq = x[m.Nu:m.off_p]
    ref = xq.copy()
    ref[fq] = spla.spsolve((tau * Mq).tocsc(), xq[fq])
    assert np.abs(y[m.Nu:m.off_p] - ref).max() < 1e-12 * np.abs(ref).max()
    assert np.all(y[:m.Nu] == 0) and np.all(y[m.off_p:] == 0)
    ctx.apply_part(B.PART_SCHUR, tau, xd, yd)
    y = yd.cpu().numpy()
    Bf = blk.B.tocsr()[:, fq]
    p = x[m.off_p:]
    beta = C2["b"] ** 2 / C2["K_dr"]
    ref = (C2["invM"] + beta) * (blk.Mp @ p) + tau * (Bf @ spla.spsolve(Mq.tocsc(), Bf.T @ p))
    assert np.abs(y[m.off_p:] - ref).max() < 1e-11 * np.abs(ref).max()


MG_CASES = [((8, 8), consolidation_bcs(2)), ((4, 4, 4), consolidation_bcs(3)), ((8, 4, 8), mixed_bcs(3))]


@pytest.mark.parametrize("n,bcs", MG_CASES)
def test_elasticity_block_and_vcycle_contraction(n, bcs):
    from paper_1801_04984_gb300 import binding as B
    rng = np.random.default_rng(22)
    K = 1e-2 * np.ones(int(np.prod(n)))
    ctx = _ctx(n, bcs, K)
    m = Mesh(n)
    blk = SpatialBlocks(m, dict(C2, K=K))
    mask = constraint_mask(m, *bcs)[: m.Nu]
    tau = 0.3
    x = np.zeros(m.N)
    x[: m.Nu] = rng.normal(size=m.Nu)
    xd = torch.tensor(x, device="cuda")
    yd = torch.empty_like(xd)
    ctx.apply_part(B.PART_ELASTICITY, tau, xd, yd)
    Md = sp.diags(mask)
    Aop = tau * (Md @ blk.A @ Md) + sp.diags(1 - mask) / 1.0
    ref = (Md @ (tau * blk.A) @ Md + sp.diags(1 - mask)) @ x[: m.Nu]
    assert np.abs(yd.cpu().numpy()[: m.Nu] - ref).max() < 1e-12 * np.abs(ref).max()
    # stationary iteration u <- u + V(b - tau A u): the V-cycle contracts the error
    b = torch.zeros_like(xd)
    b[: m.Nu] = torch.tensor(mask * rng.normal(size=m.Nu), device="cuda")
    u = torch.zeros_like(xd)
    r = b.clone()
    norms = [torch.linalg.norm(r).item()]
    for _ in range(6):
        ctx.apply_part(B.PART_VCYCLE, tau, r, yd)
        u += yd
        ctx.apply_part(B.PART_ELASTICITY, tau, u, yd)
        r = b - yd
        norms.append(torch.linalg.norm(r).item())
    rho = (norms[-1] / norms[0]) ** (1.0 / 6)
    assert rho < 0.35, norms
    del Aop


@pytest.mark.parametrize("n,bcs", CASES)
def test_lumped_schur(n, bcs):
    """Default flux-pressure block: the Darcy mass replaced by its diagonal."""
    from paper_1801_04984_gb300 import binding as B
    rng = np.random.default_rng(23)
    K = 1e-2 * np.exp(rng.normal(0, 1.5, size=int(np.prod(n))))
    ctx = _ctx(n, bcs, K, exact=0)
    m = Mesh(n)
    blk = SpatialBlocks(m, dict(C2, K=K))
    mask = constraint_mask(m, *bcs)
    fq = mask[m.Nu:m.off_p] == 1.0
    tau = 0.07
    x = rng.normal(size=m.N)
    xd = torch.tensor(x, device="cuda")
    yd = torch.empty_like(xd)
    ctx.apply_part(B.PART_SCHUR, tau, xd, yd)
    Mq = blk.Mq.tocsr()[fq][:, fq]
    Bf = blk.B.tocsr()[:, fq]
    p = x[m.off_p:]
    beta = C2["b"] ** 2 / C2["K_dr"]
    ref = (C2["invM"] + beta) * (blk.Mp @ p) + tau * (Bf @ ((Bf.T @ p) / Mq.diagonal()))
    assert np.abs(yd.cpu().numpy()[m.off_p:] - ref).max() < 1e-11 * np.abs(ref).max()


def test_fma_peak_is_measured_and_plausible():
    """biot_fma_peak: the FP32 and FP64 CUDA-core FMA throughput of this GPU (the ALU
    roofline denominators).  FP32 lies within the nominal 152 SMs x 128 lanes x 2 flop x
    clock (80.5 TFLOP/s at 2070 MHz) and is well above FP64 on this part."""
    from paper_1801_04984_gb300 import binding as B
    f32, ms32 = B.fma_peak(B.FP32)
    f64, ms64 = B.fma_peak(B.FP64)
    assert 20.0 < f32 < 85.0, f32
    assert 0.05 < f64 < f32, f64
    assert ms32 > 10.0 and ms64 > 10.0
    print("FMA peak: FP32 %.1f TFLOP/s, FP64 %.2f TFLOP/s" % (f32, f64))


@pytest.mark.parametrize("n,bcs", CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_schur_chebyshev_step_kernel(n, bcs, prec):
    """The matrix-free flux-pressure step the solver runs (weights per flux DoF, Jacobi
    diagonal formed on the fly): out = x - diag(Shat)^{-1} Shat x against the oracle's
    assembled lumped Schur complement Shat = (1/M + beta) Mp + tau B_f diag(Mq_ff)^{-1} B_f^T."""
    from paper_1801_04984_gb300 import binding as B
    rng = np.random.default_rng(29)
    K = 1e-2 * np.exp(rng.normal(0, 1.5, size=int(np.prod(n))))
    ctx = _ctx(n, bcs, K, exact=0)
    m = Mesh(n)
    blk = SpatialBlocks(m, dict(C2, K=K))
    fq = constraint_mask(m, *bcs)[m.Nu:m.off_p] == 1.0
    Mq = blk.Mq.tocsr()[fq][:, fq]
    Bf = blk.B.tocsr()[:, fq]
    beta = C2["b"] ** 2 / C2["K_dr"]
    tau = 0.07
    S = ((C2["invM"] + beta) * blk.Mp + tau * (Bf @ sp.diags(1.0 / Mq.diagonal()) @ Bf.T)).tocsr()
    dt = torch.float64 if prec == "fp64" else torch.float32
    x = rng.normal(size=m.N)
    xd = torch.tensor(x, device="cuda", dtype=dt)
    yd = torch.full_like(xd, float("nan"))
    ctx.apply_part(B.PART_SCHUR_STEP, tau, xd, yd)
    p = xd.double().cpu().numpy()[m.off_p:]
    ref = p - (S @ p) / S.diagonal()
    got = yd.double().cpu().numpy()[m.off_p:]
    tol = 1e-12 if prec == "fp64" else 2e-6
    assert np.abs(got - ref).max() < tol * np.abs(ref).max(), np.abs(got - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("n,bcs", CASES)
@pytest.mark.parametrize("tau", [0.07, 1.0])
def test_schur_spectral_bounds_and_chebyshev_degree(n, bcs, tau):
    """biot_schur_bounds on a dG(0) context against the exact spectrum of the Jacobi-scaled
    lumped Schur complement diag(Shat)^{-1} Shat (dense eigenvalues of the oracle's
    assembled Shat): the Lanczos Ritz values lie inside the spectrum (Cauchy interlacing),
    the largest one within 1 % of the largest eigenvalue, the smallest within a factor 2 of
    the smallest; the Chebyshev interval's upper end covers the spectrum; the degree is the
    one at which the Chebyshev error bound on that interval falls to ~0.07 (1.7 sqrt(kappa),
    clamped to [16, 128])."""
    import math
    from paper_1801_04984_gb300 import binding as B
    from oracle.timebasis import radau_matrices
    rng = np.random.default_rng(37)
    K = 1e-2 * np.exp(rng.normal(0, 1.5, size=int(np.prod(n))))
    ubc, fbc = bcs
    ctx = B.Context(len(n), n, dict(C2, K=K), 0, ubc, fbc)
    m = Mesh(n)
    blk = SpatialBlocks(m, dict(C2, K=K))
    fq = constraint_mask(m, *bcs)[m.Nu:m.off_p] == 1.0
    Mq = blk.Mq.tocsr()[fq][:, fq]
    Bf = blk.B.tocsr()[:, fq]
    Mt, D = radau_matrices(0)
    lam = D[0, 0] / Mt[0, 0]  # the one eigenvalue of Mt^{-1} D for dG(0)
    beta = C2["b"] ** 2 / C2["K_dr"]
    S = (lam * (C2["invM"] + beta) * blk.Mp + tau * (Bf @ sp.diags(1.0 / Mq.diagonal()) @ Bf.T)).toarray()
    d = np.diag(S)
    ev = np.linalg.eigvalsh(S / np.sqrt(np.outer(d, d)))
    ritz_lo, ritz_hi, lo, hi, deg = ctx.schur_bounds(tau)
    assert ev[0] * (1 - 1e-10) <= ritz_lo <= ritz_hi <= ev[-1] * (1 + 1e-10), (ev[0], ev[-1], ritz_lo, ritz_hi)
    assert ritz_hi > 0.99 * ev[-1] and ritz_lo < 2.0 * ev[0], (ev[0], ev[-1], ritz_lo, ritz_hi)
    assert hi >= ev[-1] and 0 < lo <= ritz_lo
    assert deg == max(16, min(128, math.ceil(1.7 * math.sqrt(hi / lo))))
