"""Generalized (implicit) leapfrog of RMHMC (oracle), Eq. leapfrog.

  p(t + e/2) = p(t) - e/2 dH/dq(q(t), p(t + e/2))                          implicit in p
  q(t + e)   = q(t) + e/2 [dH/dp(q(t), p(t+e/2)) + dH/dp(q(t+e), p(t+e/2))]  implicit in q
  p(t + e)   = p(t + e/2) - e/2 dH/dq(q(t + e), p(t + e/2))               explicit

Both implicit equations are solved by exactly n_fp fixed-point iterations each, started from
p(t) and q(t), with no early exit.
"""
import numpy as np

from .geometry import Geometry
from .softabs import G_COTH


def leapfrog(model, q, p, eps, n_fp, tau=1.0, alpha=1e6, gkind=G_COTH, geo=None):
    """One leapfrog. Returns (q_new, p_new, geometry at q_new)."""
    q = np.asarray(q, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    if geo is None:
        geo = Geometry(model, q, tau, alpha, gkind)
    ph = p.copy()
    for _ in range(n_fp):
        ph = p - 0.5 * eps * geo.dHdq(ph)
    v0 = geo.dHdp(ph)
    qn = q.copy()
    for k in range(n_fp):
        gk = geo if k == 0 else Geometry(model, qn, tau, alpha, gkind, with_third=False)
        qn = q + 0.5 * eps * (v0 + gk.dHdp(ph))
    geo_n = Geometry(model, qn, tau, alpha, gkind)
    pn = ph - 0.5 * eps * geo_n.dHdq(ph)
    return qn, pn, geo_n


def trajectory(model, q, p, eps, n_steps, n_fp, tau=1.0, alpha=1e6, gkind=G_COTH):
    """n_steps leapfrogs; returns (q, p, geometry at q, list of (q, p) after every step)."""
    geo = Geometry(model, q, tau, alpha, gkind)
    path = []
    for _ in range(n_steps):
        q, p, geo = leapfrog(model, q, p, eps, n_fp, tau, alpha, gkind, geo)
        path.append((q.copy(), p.copy()))
    return q, p, geo, path
