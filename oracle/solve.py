"""Iterative and direct solvers (oracle; test infrastructure only).

Section 2.2: a diagonal preconditioner is used and the iteration stops when
the relative residual drops below a tolerance (1e-4 in the paper).  The
paper does not name its Krylov method; the oracle uses right-preconditioned
restarted GMRES(m) (Saad & Schultz 1986) with modified Gram-Schmidt and
Givens rotations, stopping on the true residual ||b - A x|| / ||b|| <= tol.
"""

import numpy as np
import scipy.linalg


def lu_solve(Z, V):
    """Dense LU solve of Z X = V (rows of V are right-hand sides)."""
    lu = scipy.linalg.lu_factor(Z)
    return scipy.linalg.lu_solve(lu, np.atleast_2d(V).T).T


def gmres(matvec, b, diag, tol=1e-6, restart=50, maxit=2000):
    """Right-preconditioned GMRES(restart) for one right-hand side.

    ``matvec(x)`` returns A x for a vector x; ``diag`` is diag(A) and the
    preconditioner is M^-1 = diag(A)^-1, applied on the right:
    A M^-1 u = b, x = M^-1 u.  Returns (x, iterations, true relative residual).
    """
    b = np.asarray(b, dtype=np.complex128)
    dinv = 1.0 / diag
    x = np.zeros_like(b)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    it = 0
    r = b - matvec(x)
    res = np.linalg.norm(r) / bnorm
    while res > tol and it < maxit:
        beta = np.linalg.norm(r)
        m = restart
        Vb = np.zeros((m + 1, len(b)), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m, dtype=np.complex128)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        Vb[0] = r / beta
        j_end = 0
        for j in range(m):
            w = matvec(dinv * Vb[j])
            for i in range(j + 1):
                H[i, j] = np.vdot(Vb[i], w)
                w = w - H[i, j] * Vb[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                Vb[j + 1] = w / H[j + 1, j]
            # unitary rotation [[conj(c), conj(s)], [-s, c]], c = a/den, s = b/den,
            # maps (a, b) to (den, 0)
            for i in range(j):  # apply previous rotations
                t = np.conj(cs[i]) * H[i, j] + np.conj(sn[i]) * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            a, bb = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
            cs[j] = a / den if den != 0 else 1.0
            sn[j] = bb / den if den != 0 else 0.0
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = np.conj(cs[j]) * g[j]
            it += 1
            j_end = j + 1
            if abs(g[j + 1]) / bnorm <= tol or it >= maxit:
                break
        y = scipy.linalg.solve_triangular(H[:j_end, :j_end], g[:j_end])
        x = x + dinv * (y @ Vb[:j_end])
        r = b - matvec(x)
        res = np.linalg.norm(r) / bnorm
    return x, it, res
