"""Shared helpers of the GPU parity tests (problem builders; no arithmetic of the method)."""
import numpy as np

from oracle.space import F_NATURAL, F_NOFLOW, U_DIRICHLET, U_NATURAL, U_ROLLER

C1 = dict(lam=1.0, mu=1.0, b=0.9, invM=0.1, eta=1.0, K_dr=2.0)
C2 = dict(lam=1.0, mu=1.0, b=0.8, invM=0.05, eta=1.0, K_dr=1.0 + 2.0 / 3.0)


def consolidation_bcs(d):
    ubc = [U_ROLLER] * (2 * d)
    ubc[-1] = U_NATURAL
    fbc = [F_NOFLOW] * (2 * d)
    fbc[-1] = F_NATURAL
    return ubc, fbc


def dirichlet_bcs(d):
    return [U_DIRICHLET] * (2 * d), [F_NATURAL] * (2 * d)


def mixed_bcs(d):
    # every code on some face
    ubc = [U_DIRICHLET, U_ROLLER, U_NATURAL, U_ROLLER, U_ROLLER, U_NATURAL][: 2 * d]
    fbc = [F_NOFLOW, F_NATURAL, F_NOFLOW, F_NATURAL, F_NATURAL, F_NOFLOW][: 2 * d]
    return ubc, fbc
