"""Spatial matrices of the Biot system on Cartesian meshes (oracle; test
infrastructure only).

Paper §Poroelasticity (strong form) with the volumetric mean stress substituted
into the storage equation (K_dr cancels):

    -div( C:eps(u) - b p I ) = rho_b g
     eta K^{-1} q + grad p   = rho_f g
     b d_t div u + (1/M) d_t p + div q = f

Weak form, with the row signs used throughout this project:

    a(u, v) - b (p, div v)                 = (rho_b g, v) + <t_N, v>
    (eta K^{-1} q, z) - (p, div z)         = (rho_f g, z) - <p_D, z.n>
    b (div u_t, w) + (1/M)(p_t, w) + (div q, w) = (f, w)

    a(u, v) = (2 mu eps(u), eps(v)) + (lambda div u, div v)

giving the stationary part A_s = [[A, 0, -bE], [0, Mq, -B^T], [0, B, 0]] and the
storage part S = [[0,0,0],[0,0,0],[bE^T, 0, (1/M) Mp]] with

    A_ij = a(phi_j, phi_i), E_ij = (psi_j, div phi_i), Mq_ij = (eta K^{-1} z_j, z_i),
    B_ij = (div z_j, psi_i), Mp_ij = (psi_j, psi_i).

Spaces (paper §Discretisation in Space, the mixed pair Nc^f(p)-dQ(p-1) at p = 2;
the displacement is continuous Q2 here instead of the paper's interior-penalty
dG(p)):

* u: continuous Q2, Lagrange nodes {0, 1/2, 1} per cell and direction;
* q: Raviart-Thomas RT1; component c is Lagrange {0, 1/2, 1} along x_c and
  Lagrange at the two Gauss points across, normal component continuous;
* p: discontinuous Q1, Lagrange at the 2^d Gauss points of each cell.

Global DoF layout (one time level): [u_0 | .. | u_{d-1} | q_0 | .. | q_{d-1} | p],
each block a lexicographic grid with x fastest:
  u_c : (2n_x+1) x (2n_y+1) [x (2n_z+1)]
  q_c : 2n_t+1 points along direction c, 2n_t Gauss lines across each other t
  p   : (2n_x) x (2n_y) [x (2n_z)] Gauss points.

Every element matrix is computed by Gauss quadrature with 3 points per direction
(exact for all these polynomial integrands) and assembled by plain COO summation.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

G2 = np.array([0.5 - np.sqrt(3.0) / 6.0, 0.5 + np.sqrt(3.0) / 6.0])

# face / boundary condition codes
U_NATURAL, U_DIRICHLET, U_ROLLER = 0, 1, 2
F_NATURAL, F_NOFLOW = 0, 1


def q2_val(s):
    s = np.asarray(s, dtype=np.float64)
    return np.array([2.0 * (s - 0.5) * (s - 1.0), 4.0 * s * (1.0 - s), 2.0 * s * (s - 0.5)])


def q2_der(s):
    s = np.asarray(s, dtype=np.float64)
    return np.array([4.0 * s - 3.0, 4.0 - 8.0 * s, 4.0 * s - 1.0])


def g1_val(s):
    s = np.asarray(s, dtype=np.float64)
    return np.array([(s - G2[1]) / (G2[0] - G2[1]), (s - G2[0]) / (G2[1] - G2[0])])


def g1_der(s):
    s = np.asarray(s, dtype=np.float64)
    return np.array([np.full_like(s, 1.0 / (G2[0] - G2[1])), np.full_like(s, 1.0 / (G2[1] - G2[0]))])


def gauss01(npts):
    x, w = np.polynomial.legendre.leggauss(npts)
    return (x + 1.0) / 2.0, w / 2.0


def lex(idx, shape):
    """Lexicographic index with the first coordinate fastest."""
    out = 0
    mul = 1
    for i, s in zip(idx, shape):
        out = out + i * mul
        mul *= s
    return out


class Mesh:
    """Uniform Cartesian mesh of n[0] x .. x n[d-1] cells on the box [lo, hi]."""

    def __init__(self, n, lo=None, hi=None):
        self.n = tuple(int(v) for v in n)
        self.dim = len(self.n)
        assert self.dim in (2, 3)
        self.lo = np.zeros(self.dim) if lo is None else np.asarray(lo, dtype=np.float64)
        self.hi = np.ones(self.dim) if hi is None else np.asarray(hi, dtype=np.float64)
        self.h = (self.hi - self.lo) / np.array(self.n)
        d = self.dim
        self.ncells = int(np.prod(self.n))
        self.u_shape = tuple(2 * m + 1 for m in self.n)
        self.nu_nodes = int(np.prod(self.u_shape))
        self.q_shapes = [tuple((2 * self.n[t] + 1) if t == c else 2 * self.n[t] for t in range(d)) for c in range(d)]
        self.p_shape = tuple(2 * m for m in self.n)
        self.Nu = d * self.nu_nodes
        self.Nq_c = [int(np.prod(s)) for s in self.q_shapes]
        self.Nq = int(sum(self.Nq_c))
        self.Np = int(np.prod(self.p_shape))
        self.N = self.Nu + self.Nq + self.Np
        self.off_u = [c * self.nu_nodes for c in range(d)]
        self.off_q = [self.Nu + int(sum(self.Nq_c[:c])) for c in range(d)]
        self.off_p = self.Nu + self.Nq

    # ---- cells ------------------------------------------------------------
    def cells(self):
        """Array (ncells, d) of cell multi-indices in lexicographic order (x fastest)."""
        grids = np.meshgrid(*[np.arange(m) for m in self.n], indexing="ij")
        idx = np.stack([g.reshape(-1) for g in grids], axis=1)
        order = np.argsort(lex([idx[:, i] for i in range(self.dim)], self.n), kind="stable")
        return idx[order]

    # ---- local DoF sets (reference cell) ------------------------------------
    def local_u(self):
        """List of (comp, (a_0..a_{d-1})) for the 3^d Q2 nodes per component."""
        out = []
        for c in range(self.dim):
            for a in itertools.product(range(3), repeat=self.dim):
                out.append((c, a[::-1]))  # x fastest
        return out

    def local_q(self):
        """List of (comp, local index tuple): index along c in {0,1,2}, across in {0,1}."""
        out = []
        for c in range(self.dim):
            ranges = [range(3) if t == c else range(2) for t in range(self.dim)]
            for a in itertools.product(*ranges[::-1]):
                out.append((c, a[::-1]))
        return out

    def local_p(self):
        return [a[::-1] for a in itertools.product(range(2), repeat=self.dim)]

    # ---- local-to-global maps ------------------------------------------------
    def l2g(self):
        cells = self.cells()
        d = self.dim
        Lu = np.zeros((self.ncells, len(self.local_u())), dtype=np.int64)
        for j, (c, a) in enumerate(self.local_u()):
            Lu[:, j] = self.off_u[c] + lex([2 * cells[:, i] + a[i] for i in range(d)], self.u_shape)
        Lq = np.zeros((self.ncells, len(self.local_q())), dtype=np.int64)
        for j, (c, a) in enumerate(self.local_q()):
            Lq[:, j] = self.off_q[c] + lex([2 * cells[:, i] + a[i] for i in range(d)], self.q_shapes[c])
        Lp = np.zeros((self.ncells, len(self.local_p())), dtype=np.int64)
        for j, a in enumerate(self.local_p()):
            Lp[:, j] = self.off_p + lex([2 * cells[:, i] + a[i] for i in range(d)], self.p_shape)
        return cells, Lu, Lq, Lp

    # ---- basis evaluation at reference points --------------------------------
    def eval_u(self, pts):
        """Values (nloc, npts, d) and gradients (nloc, npts, d, d) [grad[..., i, j] = d_j u_i]
        of the Q2 vector basis at reference points pts (npts, d), physical scaling by h."""
        d = self.dim
        loc = self.local_u()
        V = np.zeros((len(loc), len(pts), d))
        G = np.zeros((len(loc), len(pts), d, d))
        for j, (c, a) in enumerate(loc):
            vals = [q2_val(pts[:, i])[a[i]] for i in range(d)]
            ders = [q2_der(pts[:, i])[a[i]] / self.h[i] for i in range(d)]
            V[j, :, c] = np.prod(vals, axis=0)
            for k in range(d):
                f = ders[k].copy()
                for i in range(d):
                    if i != k:
                        f = f * vals[i]
                G[j, :, c, k] = f
        return V, G

    def eval_q(self, pts):
        """Values (nloc, npts, d) and divergence (nloc, npts) of the RT1 basis."""
        d = self.dim
        loc = self.local_q()
        V = np.zeros((len(loc), len(pts), d))
        Dv = np.zeros((len(loc), len(pts)))
        for j, (c, a) in enumerate(loc):
            f = np.ones(len(pts))
            df = np.ones(len(pts))
            for i in range(d):
                if i == c:
                    f = f * q2_val(pts[:, i])[a[i]]
                    df = df * q2_der(pts[:, i])[a[i]] / self.h[i]
                else:
                    f = f * g1_val(pts[:, i])[a[i]]
                    df = df * g1_val(pts[:, i])[a[i]]
            V[j, :, c] = f
            Dv[j] = df
        return V, Dv

    def eval_p(self, pts):
        d = self.dim
        loc = self.local_p()
        V = np.zeros((len(loc), len(pts)))
        for j, a in enumerate(loc):
            f = np.ones(len(pts))
            for i in range(d):
                f = f * g1_val(pts[:, i])[a[i]]
            V[j] = f
        return V

    def quad(self, npts):
        """Tensor Gauss rule on the reference cell: points (nq, d), physical weights (nq,)."""
        x, w = gauss01(npts)
        grids = np.meshgrid(*([x] * self.dim), indexing="ij")
        wg = np.meshgrid(*([w] * self.dim), indexing="ij")
        pts = np.stack([g.reshape(-1) for g in grids], axis=1)
        W = np.prod(np.stack([g.reshape(-1) for g in wg], axis=1), axis=1) * np.prod(self.h)
        return pts, W

    # ---- element matrices ------------------------------------------------------
    def element_matrices(self, lam, mu):
        pts, W = self.quad(3)
        Vu, Gu = self.eval_u(pts)
        Vq, Dq = self.eval_q(pts)
        Vp = self.eval_p(pts)
        eps = 0.5 * (Gu + np.swapaxes(Gu, 2, 3))
        div_u = np.trace(Gu, axis1=2, axis2=3)
        A = 2.0 * mu * np.einsum("iqab,jqab,q->ij", eps, eps, W) + lam * np.einsum("iq,jq,q->ij", div_u, div_u, W)
        E = np.einsum("iq,jq,q->ij", div_u, Vp, W)
        Mq = np.einsum("iqa,jqa,q->ij", Vq, Vq, W)  # reference (unit coefficient) RT1 mass
        B = np.einsum("iq,jq,q->ij", Vp, Dq, W)
        Mp = np.einsum("iq,jq,q->ij", Vp, Vp, W)
        return A, E, Mq, B, Mp


def _coo(L_row, L_col, Ke, shape, scale=None):
    nc = L_row.shape[0]
    rows = np.repeat(L_row[:, :, None], L_col.shape[1], axis=2).reshape(-1)
    cols = np.repeat(L_col[:, None, :], L_row.shape[1], axis=1).reshape(-1)
    vals = np.broadcast_to(Ke[None], (nc,) + Ke.shape)
    if scale is not None:
        vals = vals * scale[:, None, None]
    return sp.coo_matrix((np.asarray(vals).reshape(-1), (rows, cols)), shape=shape).tocsr()


class SpatialBlocks:
    """Assembled global blocks A, E, Mq, B, Mp of one mesh and coefficient set.

    coeffs: dict with lam, mu, b, invM, eta and K (per-cell isotropic permeability,
    array of ncells, lexicographic cells)."""

    def __init__(self, mesh: Mesh, coeffs: dict):
        self.mesh = mesh
        self.coeffs = coeffs
        m = mesh
        cells, Lu, Lq, Lp = m.l2g()
        self.cells, self.Lu, self.Lq, self.Lp = cells, Lu, Lq, Lp
        A, E, Mq, B, Mp = m.element_matrices(coeffs["lam"], coeffs["mu"])
        self.Ae, self.Ee, self.Mqe, self.Be, self.Mpe = A, E, Mq, B, Mp
        # local index arrays relative to block offsets
        Lu0 = Lu
        Lq0 = Lq - m.Nu
        Lp0 = Lp - m.off_p
        self.A = _coo(Lu0, Lu0, A, (m.Nu, m.Nu))
        self.E = _coo(Lu0, Lp0, E, (m.Nu, m.Np))
        self.kscale = coeffs["eta"] / np.asarray(coeffs["K"], dtype=np.float64)
        self.Mq = _coo(Lq0, Lq0, Mq, (m.Nq, m.Nq), scale=self.kscale)
        self.B = _coo(Lp0, Lq0, B, (m.Np, m.Nq))
        self.Mp = _coo(Lp0, Lp0, Mp, (m.Np, m.Np))

    def stationary(self):
        """A_s = [[A, 0, -bE], [0, Mq, -B^T], [0, B, 0]]."""
        b = self.coeffs["b"]
        m = self.mesh
        return sp.bmat([[self.A, None, -b * self.E],
                        [None, self.Mq, -self.B.T],
                        [None, self.B, sp.csr_matrix((m.Np, m.Np))]], format="csr")

    def storage(self):
        """S = [[0,0,0],[0,0,0],[b E^T, 0, (1/M) Mp]]."""
        b, invM = self.coeffs["b"], self.coeffs["invM"]
        m = self.mesh
        return sp.bmat([[sp.csr_matrix((m.Nu, m.Nu)), None, None],
                        [None, sp.csr_matrix((m.Nq, m.Nq)), None],
                        [b * self.E.T, None, invM * self.Mp]], format="csr")


def constraint_mask(mesh: Mesh, u_bc, f_bc) -> np.ndarray:
    """1.0 for free DoFs, 0.0 for essentially constrained ones (one time level).

    Faces are numbered 2*dir + side (side 0 = lower, 1 = upper).
    u_bc[f]: U_NATURAL (traction), U_DIRICHLET (all components), U_ROLLER (normal
    component).  f_bc[f]: F_NATURAL (pressure) or F_NOFLOW (q.n = 0)."""
    d = mesh.dim
    mask = np.ones(mesh.N)
    grids = np.meshgrid(*[np.arange(s) for s in mesh.u_shape], indexing="ij")
    idx = [g.reshape(-1) for g in grids]
    lin = lex(idx, mesh.u_shape)
    for f in range(2 * d):
        dirn, side = divmod(f, 2)
        on = idx[dirn] == (0 if side == 0 else mesh.u_shape[dirn] - 1)
        for c in range(d):
            if u_bc[f] == U_DIRICHLET or (u_bc[f] == U_ROLLER and c == dirn):
                mask[mesh.off_u[c] + lin[on]] = 0.0
    for c in range(d):
        shp = mesh.q_shapes[c]
        grids = np.meshgrid(*[np.arange(s) for s in shp], indexing="ij")
        qi = [g.reshape(-1) for g in grids]
        qlin = lex(qi, shp)
        for side in range(2):
            if f_bc[2 * c + side] == F_NOFLOW:
                on = qi[c] == (0 if side == 0 else shp[c] - 1)
                mask[mesh.off_q[c] + qlin[on]] = 0.0
    return mask


def load_vector(mesh: Mesh, t: float, f_u=None, f_p=None, traction=None, p_bnd=None,
                u_bc=None, f_bc=None, nq: int = 4) -> np.ndarray:
    """Spatial load vector at time t (one time level, unmasked).

    f_u(x, t) -> (npts, d) body force rho_b g;  f_p(x, t) -> (npts,) source f;
    traction(x, t, face) -> (npts, d) on faces with natural u condition;
    p_bnd(x, t, face) -> (npts,) pressure on faces with natural flow condition
    (enters the q-rows as -<p_D, z.n>).  Gauss rule with nq points per direction."""
    m = mesh
    d = m.dim
    F = np.zeros(m.N)
    cells, Lu, Lq, Lp = m.l2g()
    pts, W = m.quad(nq)
    if f_u is not None or f_p is not None:
        X = m.lo[None, None, :] + m.h[None, None, :] * (cells[:, None, :] + pts[None, :, :])  # (nc, nq, d)
        Xf = X.reshape(-1, d)
        if f_u is not None:
            Vu, _ = m.eval_u(pts)
            fu = f_u(Xf, t).reshape(len(cells), len(pts), d)
            loc = np.einsum("jqa,cqa,q->cj", Vu, fu, W)
            np.add.at(F, Lu.reshape(-1), loc.reshape(-1))
        if f_p is not None:
            Vp = m.eval_p(pts)
            fp = f_p(Xf, t).reshape(len(cells), len(pts))
            loc = np.einsum("jq,cq,q->cj", Vp, fp, W)
            np.add.at(F, Lp.reshape(-1), loc.reshape(-1))
    if traction is not None or p_bnd is not None:
        x1, w1 = gauss01(nq)
        for f in range(2 * d):
            dirn, side = divmod(f, 2)
            others = [i for i in range(d) if i != dirn]
            grids = np.meshgrid(*([x1] * (d - 1)), indexing="ij")
            wg = np.meshgrid(*([w1] * (d - 1)), indexing="ij")
            fp_pts = np.zeros((x1.size ** (d - 1), d))
            for j, i in enumerate(others):
                fp_pts[:, i] = grids[j].reshape(-1)
            fp_pts[:, dirn] = float(side)
            fw = np.prod(np.stack([g.reshape(-1) for g in wg], axis=1), axis=1) * np.prod(m.h[others])
            sel = cells[:, dirn] == (0 if side == 0 else m.n[dirn] - 1)
            sc = cells[sel]
            X = m.lo[None, None, :] + m.h[None, None, :] * (sc[:, None, :] + fp_pts[None, :, :])
            Xf = X.reshape(-1, d)
            normal = np.zeros(d)
            normal[dirn] = -1.0 if side == 0 else 1.0
            if traction is not None and (u_bc is None or u_bc[f] == U_NATURAL):
                Vu, _ = m.eval_u(fp_pts)
                tr = traction(Xf, t, f).reshape(len(sc), len(fp_pts), d)
                loc = np.einsum("jqa,cqa,q->cj", Vu, tr, fw)
                np.add.at(F, Lu[sel].reshape(-1), loc.reshape(-1))
            if p_bnd is not None and (f_bc is None or f_bc[f] == F_NATURAL):
                Vq, _ = m.eval_q(fp_pts)
                pb = p_bnd(Xf, t, f).reshape(len(sc), len(fp_pts))
                zn = np.einsum("jqa,a->jq", Vq, normal)
                loc = -np.einsum("jq,cq,q->cj", zn, pb, fw)
                np.add.at(F, Lq[sel].reshape(-1), loc.reshape(-1))
    return F


def dofs_of_cell_rows(mesh: Mesh, gdof: int):
    """Cells (lexicographic indices) whose local DoF sets contain global DoF gdof,
    by direct index arithmetic on the DoF's grid coordinates."""
    m = mesh
    d = m.dim

    def unlex(i, shape):
        out = []
        for s in shape:
            out.append(i % s)
            i //= s
        return out

    def cells_along(k, two_n_plus_one):
        # node k on a Q2-type axis belongs to cell k//2 (if inside) and to cell k/2-1 if k even
        cs = set()
        if k // 2 < (two_n_plus_one - 1) // 2:
            cs.add(k // 2)
        if k % 2 == 0 and k > 0:
            cs.add(k // 2 - 1)
        return sorted(cs)

    if gdof < m.Nu:
        c, node = divmod(gdof, m.nu_nodes)
        co = unlex(node, m.u_shape)
        per = [cells_along(co[i], m.u_shape[i]) for i in range(d)]
    elif gdof < m.off_p:
        r = gdof - m.Nu
        c = 0
        while r >= m.Nq_c[c]:
            r -= m.Nq_c[c]
            c += 1
        co = unlex(r, m.q_shapes[c])
        per = [cells_along(co[i], m.q_shapes[c][i]) if i == c else [co[i] // 2] for i in range(d)]
    else:
        co = unlex(gdof - m.off_p, m.p_shape)
        per = [[co[i] // 2] for i in range(d)]
    return [lex(list(cc), m.n) for cc in itertools.product(*per)]
