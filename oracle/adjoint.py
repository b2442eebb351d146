"""Adjoint of the oracle's forward solve by brute force (TEST INFRASTRUCTURE
ONLY; the paper solves forward problems only, so this is the plain definition
of the gradient, not a restated algorithm).

With A the BIE matvec (kfbim.Setup.apply) and U the linear map from the
density to the velocity of the interface solve (three face fields), the
solution for boundary data g (and fixed f) has u = U A^-1 g + (terms in f),
so for a loss L(u) the gradient with respect to g is A^-T U^T dL/du.  Both A
and U are assembled column by column from unit densities with the oracle's
own forward interface solve, and the transposed system is solved densely.
Small grids only (one interface solve per density unknown).
"""
import numpy as np


# No passage: the paper solves forward problems only; A and U of the solve of Alg. 1, column by column.
def dense_maps(setup):
    """(A, U): A (n, n) with columns A e_j; U (3 N^3, n) with columns the
    interface-solve velocity of e_j, component-blocked in C order [k, j, i]."""
    n = setup.n
    N3 = setup.grid.N ** 3
    A = np.zeros((n, n))
    U = np.zeros((3 * N3, n))
    fy = np.zeros((setup.cp.n, 3))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        u, _, J = setup.interface(e, fy, None)
        A[:, j] = setup.trace(u, J)
        U[:, j] = np.concatenate([u[c].ravel() for c in range(3)])
    return A, U


# No passage: the gradient of a loss through the solve of Alg. 1 by its definition.
def gradient_g(A, U, ubar):
    """dL/dg = A^-T U^T ubar for ubar = dL/du (3 N^3)."""
    return np.linalg.solve(A.T, U.T @ ubar)
