"""SoftAbs Riemannian geometry at a point q (oracle).

Sec. 2.2: H(q) = Psi diag(lambda) Psi^T (LAPACK eigh here: an exact eigendecomposition, which the
warm-started Jacobi of Sec. 2.4 reaches up to rounding and eigenvector basis),
G(q) = Psi diag(g(lambda)) Psi^T.

Eq. Hamiltonian:  H(q, p) = U(q) + 1/2 log((2 pi)^d |G(q)|) + 1/2 p^T G(q)^-1 p.
Derivative of Eq. Hamiltonian with respect to q (the printed Eq. d_Hamiltonian has the two
metric terms with swapped signs; differentiating Eq. Hamiltonian gives):
  dH/dq_i = dU/dq_i + 1/2 tr(G^-1 dG/dq_i) - 1/2 p^T G^-1 (dG/dq_i) G^-1 p
          = dU/dq_i + 1/2 tr(W2 dH_i) - 1/2 tr(W1 dH_i)                (Eq. Betancourt_formula)
  W1 = Psi B T B Psi^T,  B = diag((Psi^T p)_j / g_j)    (= Psi ((b b^T) o T) Psi^T)
  W2 = Psi (R o T) Psi^T, R = diag(1 / g_j)               (= Psi diag(g'_j / g_j) Psi^T)
with dH_i = d/dq_i of the Hessian taken from the full third-derivative tensor.
dH/dp = G^-1 p. Momentum refresh p ~ N(0, G): p = Psi diag(sqrt g) Psi^T z (the symmetric root).
"""
from contextlib import contextmanager

import numpy as np
import scipy.linalg as sla

from . import model as mdl
from . import primal
from .softabs import G_COTH, divided_differences, g_and_gprime

LOG2PI = np.log(2.0 * np.pi)

_EIG = {"driver": "evd"}


@contextmanager
def eigen_driver(name):
    """Take the eigendecomposition of H with LAPACK's divide and conquer ('evd', numpy's eigh, the
    default) or its QR iteration ('ev'). Both are backward stable; their difference measures how
    far rounding inside any eigensolver moves the basis-free results (used to calibrate parity
    tolerances, as inverse_method does for K^-1)."""
    old = _EIG["driver"]
    _EIG["driver"] = name
    try:
        yield
    finally:
        _EIG["driver"] = old


class Geometry:
    """U, dU, Hessian, eigendecomposition and the SoftAbs metric at q (optionally with the full
    third-derivative tensor, needed for dH/dq)."""

    def __init__(self, model, q, tau=1.0, alpha=1e6, gkind=G_COTH, with_third=True):
        self.model = model
        self.q = np.array(q, dtype=np.float64)
        self.tau = tau
        self.alpha = alpha
        self.gkind = gkind
        ops = primal if isinstance(model, primal.PrimalModel) else mdl  # primal or dual GP model
        self.U = ops.potential(model, q, tau)
        self.dU = ops.gradient(model, q, tau)
        self.H = ops.hessian(model, q, tau)
        if not (np.all(np.isfinite(self.H)) and np.isfinite(self.U)):
            # a numerically failed point (Algorithm 1 rejects the proposal that reaches it); LAPACK's
            # eigensolvers are not defined on non-finite input
            raise np.linalg.LinAlgError("non-finite potential or Hessian")
        if _EIG["driver"] == "evd":
            self.lam, self.Psi = np.linalg.eigh(self.H)
        else:
            self.lam, self.Psi = sla.eigh(self.H, driver=_EIG["driver"], check_finite=False)
        self.g, self.gp = g_and_gprime(self.lam, alpha, gkind)
        self.T = divided_differences(self.lam, alpha, gkind)
        self.third = ops.ThirdDerivatives(model, q, tau).tensor() if with_third else None

    # --- metric --------------------------------------------------------------------------
    def G(self):
        return (self.Psi * self.g) @ self.Psi.T

    def logdetG(self):
        return float(np.sum(np.log(self.g)))

    def Ginv_p(self, p):
        return self.Psi @ ((self.Psi.T @ p) / self.g)

    def sqrtG_z(self, z):
        return self.Psi @ (np.sqrt(self.g) * (self.Psi.T @ z))

    def W2(self):
        return (self.Psi * (self.gp / self.g)) @ self.Psi.T

    def W1(self, p):
        b = (self.Psi.T @ p) / self.g
        return self.Psi @ (np.outer(b, b) * self.T) @ self.Psi.T

    # --- Hamiltonian ---------------------------------------------------------------------
    def hamiltonian(self, p):
        d = self.model.d
        return float(self.U + 0.5 * (d * LOG2PI + self.logdetG()) + 0.5 * p @ self.Ginv_p(p))

    def traces(self, W):
        """[tr(W dH_i)]_i over all coordinates i, from the full tensor."""
        d = self.model.d
        return self.third.reshape(d, d * d) @ W.T.reshape(d * d)

    def dHdq(self, p):
        return self.dU + 0.5 * self.traces(self.W2()) - 0.5 * self.traces(self.W1(p))

    def dHdp(self, p):
        return self.Ginv_p(p)
