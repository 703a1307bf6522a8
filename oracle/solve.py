"""Linear solves of the oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper does not name its linear solver. The oracle solves each DIA system
(Eq. 4.1) exactly where it is small: a sparse LU factorisation (SuperLU) is
used as a library step. Large systems, for which LU fill-in is prohibitive
in 3D, use conjugate gradients (pressure) or BiCGSTAB (transport) with a
Jacobi preconditioner to a tight relative residual.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .scheme import sparse_from_planes, poisson_matrix

DIRECT_MAX_ROWS = 60000
_POISSON_LU = {}


def _jacobi(A):
    d = A.diagonal().copy()
    d[d == 0.0] = 1.0
    inv = 1.0 / d
    return spla.LinearOperator(A.shape, matvec=lambda x: inv * x, dtype=np.float64)


def solve_system(planes, x0=None, method="auto", rtol=1e-14, maxiter=100000):
    """Solve the DIA system ``planes`` (with right-hand side ``planes['b']``);
    returns the solution shaped like the planes."""
    shape = planes["P"].shape
    A = sparse_from_planes(planes)
    b = planes["b"].ravel()
    if method == "auto":
        method = "direct" if A.shape[0] <= DIRECT_MAX_ROWS else "iterative"
    if method == "direct":
        x = spla.spsolve(A.tocsc(), b)
    else:
        x, info = spla.bicgstab(A, b, x0=None if x0 is None else np.ravel(x0), rtol=rtol, atol=0.0,
                                maxiter=maxiter, M=_jacobi(A))
        if info != 0:
            raise RuntimeError("oracle BiCGSTAB did not converge (info=%d)" % info)
    return x.reshape(shape)


def solve_poisson(grid, b, method="auto", rtol=1e-14, maxiter=200000):
    """Solve A p' = b with A = -L (Neumann Laplacian) for the zero-mean p'.

    ``b`` must have zero mean (consistent system). The direct path fixes the
    gauge by replacing the first equation with p'_0 = 0, which is exact for a
    consistent system because the equations sum to zero, then removes the
    mean. The iterative path runs CG from 0 and removes the mean."""
    A = sparse_from_planes(poisson_matrix(grid))
    n = A.shape[0]
    bv = np.ravel(b).copy()
    if method == "auto":
        method = "direct" if n <= DIRECT_MAX_ROWS else "iterative"
    if method == "direct":
        key = grid.key()
        lu = _POISSON_LU.get(key)
        if lu is None:
            Ap = A.tolil()
            Ap[0, :] = 0.0
            Ap[0, 0] = 1.0
            lu = spla.splu(Ap.tocsc())
            if len(_POISSON_LU) > 16:
                _POISSON_LU.clear()
            _POISSON_LU[key] = lu
        bv[0] = 0.0
        x = lu.solve(bv)
    else:
        x, info = spla.cg(A, bv, rtol=rtol, atol=0.0, maxiter=maxiter, M=_jacobi(A))
        if info != 0:
            raise RuntimeError("oracle CG did not converge (info=%d)" % info)
    x = x - x.mean()
    return x.reshape(grid.cells)
