"""FP64 oracle of the zero-fill incomplete Cholesky preconditioner, IC(0),
for the PCG solve of Eq. 13.

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU leg).  Sec. III
preconditions the conjugate gradients with an incomplete Cholesky
factorisation; the paper does not state the variant, and this is the
zero-fill one: L lower triangular on the pattern of tril(A) with

    (L L^T)_ij = A_ij  for every (i, j) in the pattern of A,

computed row by row in increasing index order:

    L_ij = (A_ij - sum_k L_ik L_jk) / L_jj    for j < i in the pattern of row i
    L_ii = sqrt(A_ii - sum_{j < i} L_ij^2)

where k runs over the columns below j present in the patterns of both rows
i and j.  For an M-matrix (the system matrix lambda (D2 - W o W) + r D is
one) every pivot is positive (Meijerink and van der Vorst, 1977).  The
preconditioner is M^{-1} = L^{-T} L^{-1}.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def ic0(A: sp.spmatrix) -> sp.csr_matrix:
    """The IC(0) factor L (CSR, lower triangular with the diagonal)."""
    A = sp.csr_matrix(A, dtype=np.float64)
    A.sort_indices()
    n = A.shape[0]
    rows = []  # per row: dict column -> value of L (columns <= i)
    for i in range(n):
        cols = A.indices[A.indptr[i]:A.indptr[i + 1]]
        vals = A.data[A.indptr[i]:A.indptr[i + 1]]
        li = {}
        diag = None
        for j, a in zip(cols, vals):
            if j > i:
                break
            if j == i:
                diag = a
                break
            lj = rows[j]
            s = a
            for k, lik in li.items():  # k < j: columns of row i already computed
                ljk = lj.get(k)
                if ljk is not None:
                    s -= lik * ljk
            li[j] = s / lj[j]
        if diag is None:
            raise ValueError("zero diagonal in row %d" % i)
        piv = diag - sum(v * v for v in li.values())
        if not piv > 0.0:
            raise ValueError("non-positive pivot %g in row %d" % (piv, i))
        li[i] = np.sqrt(piv)
        rows.append(li)
    indptr = np.zeros(n + 1, dtype=np.int64)
    for i, li in enumerate(rows):
        indptr[i + 1] = indptr[i] + len(li)
    indices = np.empty(indptr[-1], dtype=np.int64)
    data = np.empty(indptr[-1])
    for i, li in enumerate(rows):
        ks = sorted(li)
        indices[indptr[i]:indptr[i + 1]] = ks
        data[indptr[i]:indptr[i + 1]] = [li[k] for k in ks]
    return sp.csr_matrix((data, indices, indptr), shape=(n, n))


def ic0_apply(L: sp.csr_matrix, R: np.ndarray) -> np.ndarray:
    """z = L^{-T} (L^{-1} r), column by column."""
    Y = spla.spsolve_triangular(L, R, lower=True)
    return spla.spsolve_triangular(sp.csr_matrix(L.T), Y, lower=False)
