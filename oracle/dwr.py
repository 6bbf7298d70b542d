"""Goal-oriented (dual-weighted residual) estimate of the time-discretisation error
(oracle; test infrastructure only).

Paper §Abstract: variational space-time methods allow goal-oriented, duality-based
adaptivity.  For J(U) = j^T U(T^-) the error of the dG(r) solution in time is estimated
against dG(r+1): the degree-r slab polynomials are degree-(r+1) polynomials whose top
Legendre mode vanishes, so the dG(r) slab solution X_n embeds into the dG(r+1) system as
Y_n = [X_n; 0] (Legendre basis).  With the dG(r+1) dual solution Z_n (calA^T Z_N = phi(1) j,
calA^T Z_n = C^T Z_{n+1}) the slab indicators are

    eta_n = Z_n^T ( F_n + C Y_{n-1} - calA Y_n ),

and since the slab systems form one block-bidiagonal linear system, their sum equals
J(U_{r+1}) - J(U_r) exactly (the dual pairs the error of the embedded solution with the
residual).  The indicators show which slabs carry the error of the goal.
"""
from __future__ import annotations

import numpy as np

from .slab import SlabProblem


def dwr_time_indicators(prob_r: SlabProblem, prob_r1: SlabProblem, T: float, slabs: int, load_fn, j_end,
                        U0=None):
    """Returns (eta_n for every slab, J(U_r))."""
    assert prob_r1.r == prob_r.r + 1 and prob_r1.N == prob_r.N
    Xs, U_end = prob_r.march(T, slabs, load_fn, U0)
    Zs = prob_r1.adjoint_march(T, slabs, None, j_end)
    tau = T / slabs
    A1 = prob_r1.operator(tau)
    N = prob_r.N
    U = np.zeros(N) if U0 is None else np.asarray(U0, dtype=np.float64).copy()
    eta = []
    for n in range(slabs):
        Y = np.concatenate([Xs[n], np.zeros(N)])  # top Legendre mode of degree r+1 is zero
        rhs = prob_r1.mask * prob_r1.slab_load(tau, n * tau, load_fn) + prob_r1.jump_rhs(U)
        eta.append(float(Zs[n] @ (rhs - A1 @ Y)))
        U = prob_r.end_value(Xs[n])
    return np.array(eta), float(j_end @ U_end)
