"""Linear algebra of the oracle.  TEST INFRASTRUCTURE ONLY.

* CGNR: conjugate gradients on the normal equations D^dagger D x = D^dagger b,
  textbook form (Hestenes-Stiefel), with a restart on the true residual so
  that the returned x satisfies |b - D x| <= tol |b| whenever it reports
  convergence.  The paper leaves the solver open ("inversions", Sec. 5); any
  solver meeting the residual gives the same x up to that residual.
* LU with partial pivoting for log|det| of small dense matrices (the paper's
  exact small-block determinants, Sec. 3, use a sparse LU).
"""
import numpy as np


def vdot(a, b):
    return np.vdot(a.reshape(-1), b.reshape(-1))


def norm2(a):
    return float(np.real(vdot(a, a)))


def cgnr(apply, apply_dag, b, tol=1e-13, maxit=100000, x0=None):
    """Solve D x = b.  Returns (x, iterations, true relative residual)."""
    bb = norm2(b)
    if bb == 0.0:
        return np.zeros_like(b), 0, 0.0
    x = np.zeros_like(b) if x0 is None else x0.copy()
    it = 0
    while True:
        r = b - apply(x)
        rel = np.sqrt(norm2(r) / bb)
        if rel <= tol or it >= maxit:
            return x, it, rel
        z = apply_dag(r)
        p = z.copy()
        zz = norm2(z)
        target = (0.1 * tol) ** 2 * bb
        while it < maxit:
            q = apply(p)
            alpha = zz / norm2(q)
            x = x + alpha * p
            r = r - alpha * q
            it += 1
            if norm2(r) <= target:
                break
            z = apply_dag(r)
            zz_new = norm2(z)
            p = z + (zz_new / zz) * p
            zz = zz_new


def lu_logabsdet(A):
    """log|det A| by Gaussian elimination with partial pivoting."""
    A = np.array(A, dtype=np.complex128, copy=True)
    n = A.shape[0]
    logdet = 0.0
    for k in range(n):
        p = k + int(np.argmax(np.abs(A[k:, k])))
        if A[p, k] == 0:
            return -np.inf
        if p != k:
            A[[k, p]] = A[[p, k]]
        piv = A[k, k]
        logdet += np.log(abs(piv))
        if k + 1 < n:
            f = A[k + 1:, k] / piv
            A[k + 1:, k + 1:] -= np.outer(f, A[k, k + 1:])
    return logdet
