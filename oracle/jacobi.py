"""Cyclic Jacobi eigensolver with sweep counting (oracle; used only for the sweep-count checks of
Sec. 2.4 / Sec. 3.1, never for the oracle's own geometry, which uses LAPACK eigh).

Sec. 2.4: with Psi from the previous point, M = Psi^T H Psi is diagonal up to O(eps); cyclic Jacobi
drives its off-diagonal part to the tolerance zeta, M = Q diag(lambda) Q^T, and Psi <- Psi Q.
Stopping rule (the tolerance zeta is not defined further in Sec. 2.4; relative reading): sweeps
continue while some |m_jl| > max(zeta sqrt(|m_jj m_ll|), 4 u ||M||_F) (u = 2^-53; the floor is
the rounding level rotations leave behind), checked before every sweep (an already diagonal M
takes 0 sweeps), up to max_sweeps; the Frobenius reading ||offdiag||_F > zeta ||M||_F is
available as rule='frobenius'.
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


U_ROUND = 2.0 ** -53


def relative_offdiag(M, tol, rule="relative"):
    """max over j != l of |m_jl| / max(tol * den_jl, 4 u ||M||_F); <= 1 is converged.
    den_jl = sqrt(|m_jj m_ll|) ('relative') or |m_jj m_ll| / min_i |m_ii| ('metric')."""
    d = np.abs(np.diag(M))
    floor = 4.0 * U_ROUND * np.linalg.norm(M)
    if rule == "metric":
        den = np.outer(d, d) / max(d.min(), 1e-300)
    else:
        den = np.sqrt(np.outer(d, d))
    den = np.maximum(tol * den, max(floor, 1e-300))
    R = np.abs(M) / den
    np.fill_diagonal(R, 0.0)
    return float(R.max()) if R.size else 0.0


def jacobi_eigh(H, Psi0=None, tol=1e-13, max_sweeps=30, rule="relative"):
    """Returns (lam, Psi, sweeps). Psi0 = None is the cold start Psi0 = I.
    rule 'relative': continue while some |m_jl| > max(tol sqrt(|m_jj m_ll|), 4 u ||M||_F);
    rule 'metric': continue while some |m_jl| > max(tol |m_jj m_ll| / min_i |m_ii|, 4 u ||M||_F)
    (the coupling's first-order effect on G^-1 below tol relative); rule 'frobenius': continue
    while ||offdiag(M)||_F > tol ||M||_F."""
    H = np.asarray(H, dtype=np.float64)
    d = H.shape[0]
    Psi = np.eye(d) if Psi0 is None else np.array(Psi0, dtype=np.float64)
    M = Psi.T @ H @ Psi
    M = 0.5 * (M + M.T)
    sweeps = 0
    def unconverged(M):
        if rule == "frobenius":
            return offdiag_norm(M) > tol * np.linalg.norm(M)
        return relative_offdiag(M, tol, rule) > 1.0

    while unconverged(M) and sweeps < max_sweeps:
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
