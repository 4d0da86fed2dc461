"""Cyclic Jacobi eigensolver with sweep counting (oracle; used only for the sweep-count checks of
Sec. 2.4 / Sec. 3.1, never for the oracle's own geometry, which uses LAPACK eigh).

Sec. 2.4: with Psi from the previous point, M = Psi^T H Psi is diagonal up to O(eps); cyclic Jacobi
drives its off-diagonal part to the tolerance zeta, M = Q diag(lambda) Q^T, and Psi <- Psi Q.
Stopping rule: sweeps continue while ||offdiag(M)||_F > zeta ||M||_F (checked before every sweep,
so an already-diagonal M takes 0 sweeps), up to max_sweeps.
Each rotation is the symmetric 2x2 Schur decomposition (Golub and Van Loan, "Matrix
Computations", Sec. 8.5): for the pair (j, l) with M_jl != 0,
  theta = (M_ll - M_jj) / (2 M_jl),  t = sign(theta) / (|theta| + sqrt(1 + theta^2)),
  c = 1 / sqrt(1 + t^2),  s = t c,   J = [[c, s], [-s, c]] on (j, l),  M <- J^T M J,  Q <- Q J.
"""
import numpy as np


def offdiag_norm(M):
    """Frobenius norm of the off-diagonal part (summed directly: subtracting the diagonal's
    squares from ||M||_F^2 would cancel down to ~sqrt(eps) ||M||_F)."""
    off = M - np.diag(np.diag(M))
    return float(np.sqrt(np.sum(off * off)))


def jacobi_eigh(H, Psi0=None, tol=1e-13, max_sweeps=30):
    """Returns (lam, Psi, sweeps). Psi0 = None is the cold start Psi0 = I."""
    H = np.asarray(H, dtype=np.float64)
    d = H.shape[0]
    Psi = np.eye(d) if Psi0 is None else np.array(Psi0, dtype=np.float64)
    M = Psi.T @ H @ Psi
    M = 0.5 * (M + M.T)
    sweeps = 0
    while offdiag_norm(M) > tol * np.linalg.norm(M) and sweeps < max_sweeps:
        for j in range(d - 1):
            for l in range(j + 1, d):
                mjl = M[j, l]
                if mjl == 0.0:
                    continue
                theta = (M[l, l] - M[j, j]) / (2.0 * mjl)
                if theta == 0.0:
                    t = 1.0
                elif abs(theta) > 1e150:
                    t = 0.5 / theta
                else:
                    t = np.sign(theta) / (abs(theta) + np.sqrt(1.0 + theta * theta))
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = t * c
                Mj = M[j, :].copy()
                Ml = M[l, :].copy()
                M[j, :] = c * Mj - s * Ml
                M[l, :] = s * Mj + c * Ml
                Mj = M[:, j].copy()
                Ml = M[:, l].copy()
                M[:, j] = c * Mj - s * Ml
                M[:, l] = s * Mj + c * Ml
                M[j, l] = M[l, j] = 0.0
                Pj = Psi[:, j].copy()
                Pl = Psi[:, l].copy()
                Psi[:, j] = c * Pj - s * Pl
                Psi[:, l] = s * Pj + c * Pl
        sweeps += 1
    return np.diag(M).copy(), Psi, sweeps
