"""Monolithic space-time slab system, direct solves, marching and the adjoint
(oracle; test infrastructure only).

Paper §Monolithic Approach: on each slab the coupled system for all r+1 temporal
DoFs (u^j, q^j, p^j) is assembled and solved at once; slabs are marched in time
(§Discretisation in Time).  With the semi-discrete form S U' + A_s U = F (see
`oracle.space`) and the time matrices of `oracle.timebasis`,

    calA = D (x) S + tau M_t (x) A_s          (time-major Kronecker layout)
    calA X_n = F_n + (phi(0) phi(1)^T (x) S) X_{n-1}
    F_{n,k}  = int_{I_n} phi_k((t - t_{n-1})/tau) F(t) dt.

Essential conditions: with the 0/1 free mask M (all temporal levels),
calA_c = M calA M + (I - M) and rhs_c = M rhs (homogeneous data only).

The solve is a sparse direct LU (scipy SuperLU), in the Legendre time basis
unless `basis='radau'` is asked for.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import timebasis as tb
from .space import Mesh, SpatialBlocks, constraint_mask, gauss01, lex, g1_val


class SlabProblem:
    def __init__(self, mesh: Mesh, coeffs: dict, r: int, u_bc, f_bc):
        self.mesh = mesh
        self.coeffs = coeffs
        self.r = int(r)
        self.u_bc = list(u_bc)
        self.f_bc = list(f_bc)
        self.blocks = SpatialBlocks(mesh, coeffs)
        self.As = self.blocks.stationary()
        self.S = self.blocks.storage()
        self.mask1 = constraint_mask(mesh, u_bc, f_bc)
        self.mask = np.tile(self.mask1, self.r + 1)
        self.N = mesh.N
        self.Nslab = mesh.N * (self.r + 1)

    # ---- time matrices ---------------------------------------------------------
    def time_mats(self, basis):
        return tb.legendre_matrices(self.r) if basis == "legendre" else tb.radau_matrices(self.r)

    def phi(self, s, basis):
        return tb.basis_values(np.atleast_1d(s), self.r, basis)

    # ---- operator ----------------------------------------------------------------
    def operator(self, tau: float, basis: str = "legendre", masked: bool = True) -> sp.csr_matrix:
        Mt, D = self.time_mats(basis)
        A = sp.kron(sp.csr_matrix(D), self.S) + tau * sp.kron(sp.csr_matrix(Mt), self.As)
        A = A.tocsr()
        if not masked:
            return A
        Md = sp.diags(self.mask)
        return (Md @ A @ Md + sp.diags(1.0 - self.mask)).tocsr()

    def coupling(self, basis: str = "legendre") -> sp.csr_matrix:
        """C with rhs_n += C X_{n-1}: (phi(0) phi(1)^T) (x) S, rows masked."""
        p0 = self.phi(0.0, basis)[:, 0]
        p1 = self.phi(1.0, basis)[:, 0]
        C = sp.kron(sp.csr_matrix(np.outer(p0, p1)), self.S).tocsr()
        return (sp.diags(self.mask) @ C).tocsr()

    # ---- loads --------------------------------------------------------------------
    def slab_load(self, tau: float, t0: float, load_fn, basis: str = "legendre", nt: int = 8) -> np.ndarray:
        """F_k = tau int_0^1 phi_k(s) F(t0 + tau s) ds by nt-point Gauss in time."""
        F = np.zeros(self.Nslab)
        if load_fn is None:
            return F
        s, w = gauss01(nt)
        ph = self.phi(s, basis)
        for q in range(nt):
            Fq = load_fn(t0 + tau * s[q])
            for k in range(self.r + 1):
                F[k * self.N:(k + 1) * self.N] += tau * w[q] * ph[k, q] * Fq
        return F

    def end_value(self, X: np.ndarray, basis: str = "legendre") -> np.ndarray:
        p1 = self.phi(1.0, basis)[:, 0]
        Xk = X.reshape(self.r + 1, self.N)
        return p1 @ Xk

    def value_at(self, X: np.ndarray, s: float, basis: str = "legendre") -> np.ndarray:
        ps = self.phi(s, basis)[:, 0]
        return ps @ X.reshape(self.r + 1, self.N)

    # ---- solves -------------------------------------------------------------------
    def factor(self, tau: float, basis: str = "legendre"):
        return spla.splu(self.operator(tau, basis).tocsc())

    def jump_rhs(self, U_prev_end: np.ndarray, basis: str = "legendre") -> np.ndarray:
        """phi_k(0) S U(t_{n-1}^-) for every k (masked)."""
        p0 = self.phi(0.0, basis)[:, 0]
        SU = self.S @ U_prev_end
        return self.mask * np.concatenate([p0[k] * SU for k in range(self.r + 1)])

    def march(self, T: float, slabs: int, load_fn, U0=None, basis: str = "legendre", t_start: float = 0.0):
        """Returns (list of slab solutions X_n, U(T^-))."""
        tau = (T - t_start) / slabs
        lu = self.factor(tau, basis)
        U = np.zeros(self.N) if U0 is None else np.asarray(U0, dtype=np.float64).copy()
        Xs = []
        for n in range(slabs):
            t0 = t_start + n * tau
            rhs = self.mask * self.slab_load(tau, t0, load_fn, basis) + self.jump_rhs(U, basis)
            X = lu.solve(rhs)
            Xs.append(X)
            U = self.end_value(X, basis)
        return Xs, U

    # ---- adjoint -------------------------------------------------------------------
    def adjoint_march(self, T: float, slabs: int, Xs, j_end: np.ndarray, basis: str = "legendre"):
        """Adjoint states Z_n for J = j_end^T U(T^-):
        calA^T Z_N = phi(1) (x) j_end,  calA^T Z_n = C^T Z_{n+1}."""
        tau = T / slabs
        At = self.operator(tau, basis).T.tocsc()
        lu = spla.splu(At)
        C = self.coupling(basis)
        p1 = self.phi(1.0, basis)[:, 0]
        Zs = [None] * slabs
        rhs = np.concatenate([p1[k] * j_end for k in range(self.r + 1)])
        for n in range(slabs - 1, -1, -1):
            if n < slabs - 1:
                rhs = C.T @ Zs[n + 1]
            Zs[n] = lu.solve(rhs)
        return Zs

    def grad_logk(self, T: float, slabs: int, Xs, Zs, basis: str = "legendre") -> np.ndarray:
        """dJ/dg_c for K_c = K0 exp(g_c):  sum_n sum_kl tau (M_t)_kl (eta/K_c)
        (M Z_{n,k})_c^T Mq_ref (M X_{n,l})_c, from dcalA/dg_c = -tau M_t (x) (eta/K_c) Mq_ref_c."""
        tau = T / slabs
        Mt, _ = self.time_mats(basis)
        blk = self.blocks
        m = self.mesh
        kscale = blk.kscale
        Lq = blk.Lq  # global indices (one level)
        g = np.zeros(m.ncells)
        for n in range(len(Xs)):
            X = (self.mask * Xs[n]).reshape(self.r + 1, self.N)
            Z = (self.mask * Zs[n]).reshape(self.r + 1, self.N)
            for k in range(self.r + 1):
                zc = Z[k][Lq]  # (ncells, nloc)
                for l in range(self.r + 1):
                    if Mt[k, l] == 0.0:
                        continue
                    xc = X[l][Lq]
                    g += tau * Mt[k, l] * kscale * np.einsum("ci,ij,cj->c", zc, blk.Mqe, xc)
        return g

    # ---- checks -------------------------------------------------------------------
    def residual(self, X, rhs, tau, basis="legendre"):
        return rhs - self.operator(tau, basis) @ X


def goal_vector_mean_p(mesh: Mesh, box_lo, box_hi) -> np.ndarray:
    """j with j^T U = (1/|box|) int_box p dx, exact for DGQ1 p (Gauss rule on the
    clipped part of every cell)."""
    d = mesh.dim
    j = np.zeros(mesh.N)
    vol = float(np.prod(np.asarray(box_hi) - np.asarray(box_lo)))
    xg, wg = gauss01(3)
    cells = mesh.cells()
    for ci, cell in enumerate(cells):
        lo_c = mesh.lo + mesh.h * cell
        hi_c = lo_c + mesh.h
        a = np.maximum(lo_c, box_lo)
        b = np.minimum(hi_c, box_hi)
        if np.any(b <= a):
            continue
        # 1-D integrals of the two Gauss-Lagrange functions over [a_i, b_i]
        I = []
        for i in range(d):
            sa = (a[i] - lo_c[i]) / mesh.h[i]
            sb = (b[i] - lo_c[i]) / mesh.h[i]
            s = sa + (sb - sa) * xg
            I.append((g1_val(s) @ wg) * (sb - sa) * mesh.h[i])
        for gi in np.ndindex(*([2] * d)):
            g = gi[::-1]
            val = np.prod([I[i][g[i]] for i in range(d)])
            idx = mesh.off_p + lex([2 * cell[i] + g[i] for i in range(d)], mesh.p_shape)
            j[idx] += val / vol
    return j


class CellwiseSlab:
    """What `apply_rows` needs of a slab problem, without any global assembly: the
    local-to-global maps, the reference element matrices, the per-cell Darcy factor
    eta/K_c, the constraint mask of one time level and the time matrices.  Used at
    sizes where the assembled slab matrix of `SlabProblem` does not fit in memory
    (paper §Monolithic Approach: the same slab operator, evaluated row by row)."""

    def __init__(self, mesh: Mesh, coeffs: dict, r: int, u_bc, f_bc):
        from types import SimpleNamespace
        self.mesh = mesh
        self.coeffs = coeffs
        self.r = int(r)
        cells, Lu, Lq, Lp = mesh.l2g()
        A, E, Mq, B, Mp = mesh.element_matrices(coeffs["lam"], coeffs["mu"])
        kscale = coeffs["eta"] / np.asarray(coeffs["K"], dtype=np.float64)
        self.blocks = SimpleNamespace(Lu=Lu, Lq=Lq, Lp=Lp, Ae=A, Ee=E, Mqe=Mq, Be=B, Mpe=Mp, kscale=kscale)
        self.mask1 = constraint_mask(mesh, u_bc, f_bc)
        self.N = mesh.N
        self.Nslab = mesh.N * (self.r + 1)

    def time_mats(self, basis):
        return tb.legendre_matrices(self.r) if basis == "legendre" else tb.radau_matrices(self.r)


def apply_rows(prob, tau: float, X: np.ndarray, rows, basis: str = "radau") -> np.ndarray:
    """Selected entries of calA_c X computed cell by cell from the element matrices
    (no global assembly), for parity checks at sizes where the sparse slab matrix
    does not fit: y_(k,i) = sum_l D_kl (S X_l)_i + tau (M_t)_kl (A_s X_l)_i on free
    rows, y = X on constrained rows.  `prob` is a SlabProblem or a CellwiseSlab."""
    from .space import dofs_of_cell_rows
    m = prob.mesh
    blk = prob.blocks
    b, invM = prob.coeffs["b"], prob.coeffs["invM"]
    Mt, D = prob.time_mats(basis)
    N = m.N
    nu, nq, npl = blk.Lu.shape[1], blk.Lq.shape[1], blk.Lp.shape[1]
    Xm = X.reshape(prob.r + 1, N) * prob.mask1[None, :]
    out = np.zeros(len(rows))
    for ri, row in enumerate(rows):
        k, i = divmod(int(row), N)
        if prob.mask1[i] == 0.0:
            out[ri] = X[row]
            continue
        acc = 0.0
        for c in dofs_of_cell_rows(m, i):
            L = np.concatenate([blk.Lu[c], blk.Lq[c], blk.Lp[c]])
            loc = int(np.nonzero(L == i)[0][0])
            As = np.zeros((len(L), len(L)))
            Se = np.zeros((len(L), len(L)))
            As[:nu, :nu] = blk.Ae
            As[:nu, nu + nq:] = -b * blk.Ee
            As[nu:nu + nq, nu:nu + nq] = blk.kscale[c] * blk.Mqe
            As[nu:nu + nq, nu + nq:] = -blk.Be.T
            As[nu + nq:, nu:nu + nq] = blk.Be
            Se[nu + nq:, :nu] = b * blk.Ee.T
            Se[nu + nq:, nu + nq:] = invM * blk.Mpe
            for l in range(prob.r + 1):
                xl = Xm[l][L]
                acc += D[k, l] * (Se[loc] @ xl) + tau * Mt[k, l] * (As[loc] @ xl)
        out[ri] = acc
    return out
