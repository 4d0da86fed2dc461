"""Algorithm 1, (RM)HMC with Metropolis-Hastings (oracle).

Per iteration l (global index, counted from 0 across burn-in and recorded iterations):
  z ~ N(0, I) from Philox (key (seed, chain), counter (block, l, 0, 0)); p = G(q)^{1/2} z
  H0 = H(q, p); C leapfrogs -> (q*, p*); H1 = H(q*, p*)
  r ~ U[0, 1) (counter (0, l, 1, 0)); accept iff log r < H0 - H1 (and H1 finite), else keep q.
The printed test of Algorithm 1 reads as the reverse branch; standard Metropolis-Hastings
(accept with probability min(1, exp(H0 - H1))) is what the sampler must do to target P.
The momentum is redrawn at every iteration, which is Algorithm 1's initial draw followed by
its draw after every Metropolis-Hastings step.
A trajectory that fails numerically (a kernel matrix that is not positive definite, a non-finite
value) is a rejected proposal: the chain keeps q, and H1 is recorded as +inf.
"""
import numpy as np

from .geometry import Geometry
from .integrator import leapfrog
from .philox import mh_uniform, normals
from .softabs import G_COTH


def sample(model, q0, n_iter, n_burn, seed, chain, eps, n_leapfrog, n_fp, tau=1.0, alpha=1e6,
           gkind=G_COTH, iter_offset=0):
    """Returns dict with q (n_iter x d), logp (n_iter), accept (n_iter), H0/H1 per iteration."""
    d = model.d
    q = np.array(q0, dtype=np.float64)
    geo = Geometry(model, q, tau, alpha, gkind)
    out_q, out_lp, out_acc, out_h0, out_h1 = [], [], [], [], []
    for it in range(n_burn + n_iter):
        l = iter_offset + it
        z = normals(seed, chain, l, d)
        p = geo.sqrtG_z(z)
        H0 = geo.hamiltonian(p)
        qn, pn, gn = q, p, geo
        try:
            with np.errstate(all="ignore"):
                for _ in range(n_leapfrog):
                    qn, pn, gn = leapfrog(model, qn, pn, eps, n_fp, tau, alpha, gkind, gn)
                H1 = gn.hamiltonian(pn)
        except np.linalg.LinAlgError:
            H1 = np.inf
        r = mh_uniform(seed, chain, l)
        with np.errstate(divide="ignore"):
            logr = np.log(r)
        acc = bool(np.isfinite(H1) and logr < H0 - H1)
        if acc:
            q, geo = qn, gn
        if it >= n_burn:
            out_q.append(q.copy())
            out_lp.append(-geo.U)
            out_acc.append(acc)
            out_h0.append(H0)
            out_h1.append(H1)
    return {"q": np.array(out_q), "logp": np.array(out_lp), "accept": np.array(out_acc),
            "H0": np.array(out_h0), "H1": np.array(out_h1)}
