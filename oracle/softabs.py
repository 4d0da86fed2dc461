"""Soft-absolute eigenvalue map and the divided-difference matrix T (oracle).

Sec. 2.2: the Hessian H = sum_i lambda_i psi_i psi_i^T becomes the metric
G = sum_i g(lambda_i) psi_i psi_i^T with g(lambda) ~ |lambda|. Two maps are supported:

  coth (Betancourt):  g(l) = l * coth(alpha l),    g'(l) = coth(alpha l) - alpha l / sinh^2(alpha l)
  sqrt (Sec. 2.5):    g(l) = sqrt(kappa^2 + l^2),  g'(l) = l / sqrt(kappa^2 + l^2)

coth is singular at 0 as written (the paper's reason for avoiding it, Sec. 2.5). With x = alpha l
the oracle evaluates it piecewise:
  g : |x| < 1e-3  Laurent series x coth x = 1 + x^2/3 - x^4/45 + 2 x^6/945, g = (x coth x) / alpha
      |x| > 20    coth x = sign(x) to double precision, g = |l|
      otherwise   g = l / tanh(x)
  g': |x| < 1e-3  g' = d(x coth x)/dx = 2x/3 - 4x^3/45 + 4x^5/315
      |x| <= 1    g' = (sinh(2x) - 2x) / (2 sinh(x)^2), with sinh(y) - y = sum_{k>=1} y^(2k+1)/(2k+1)!
                  summed to k = 12 (all terms one sign: no cancellation; the direct
                  coth x - x / sinh^2 x loses ~1.5 / x^2 ulps here)
      |x| > 20    g' = sign(l)
      otherwise   g' = 1/tanh(x) - x / sinh(x)^2
so g(0) = 1/alpha and g'(0) = 0.

T (Eq. d3_transform): T_jl = (g(l_j) - g(l_l)) / (l_j - l_l) for distinct eigenvalues and g'(l_j)
on the diagonal. Near-equal eigenvalues, |l_j - l_l| <= 1e-7 * max(1, |l_j|, |l_l|), take the
limit value g'((l_j + l_l) / 2) (symmetric in j, l; equal to g'(l_j) when l_j = l_l exactly).
"""
import numpy as np

G_COTH = "coth"
G_SQRT = "sqrt"
SERIES_X = 1e-3
SATURATE_X = 20.0
SINH_SERIES_X = 1.0
SINH_SERIES_TERMS = 12
NEAR_EQUAL = 1e-7


def _sinh_minus_identity(y):
    """sinh(y) - y = sum_{k=1..12} y^(2k+1) / (2k+1)!  (Taylor series of sinh; |y| <= 2)."""
    y2 = y * y
    acc = np.zeros_like(y)
    for k in range(SINH_SERIES_TERMS, 0, -1):
        acc = acc * y2 + 1.0 / float(np.prod(np.arange(1, 2 * k + 2, dtype=np.float64)))
    return acc * y2 * y


def g_and_gprime(lam, alpha=1e6, kind=G_COTH):
    """Element-wise g(lambda), g'(lambda). For kind 'sqrt', alpha is 1/kappa."""
    lam = np.asarray(lam, dtype=np.float64)
    if kind == G_SQRT:
        kappa = 1.0 / alpha
        r = np.sqrt(kappa * kappa + lam * lam)
        return r, lam / r
    x = alpha * lam
    ax = np.abs(x)
    g = np.empty_like(lam)
    gp = np.empty_like(lam)
    small = ax < SERIES_X
    big = ax > SATURATE_X
    mid = ~(small | big)
    xs = x[small]
    x2 = xs * xs
    g[small] = (1.0 + x2 / 3.0 - x2 * x2 / 45.0 + 2.0 * x2 ** 3 / 945.0) / alpha
    gp[small] = 2.0 * xs / 3.0 - 4.0 * xs * x2 / 45.0 + 4.0 * xs * x2 * x2 / 315.0
    g[big] = np.abs(lam[big])
    gp[big] = np.sign(lam[big])
    xm = x[mid]
    th = np.tanh(xm)
    sh = np.sinh(xm)
    g[mid] = lam[mid] / th
    gpm = 1.0 / th - xm / (sh * sh)
    near0 = np.abs(xm) <= SINH_SERIES_X
    gpm[near0] = _sinh_minus_identity(2.0 * xm[near0]) / (2.0 * sh[near0] * sh[near0])
    gp[mid] = gpm
    return g, gp


def divided_differences(lam, alpha=1e6, kind=G_COTH):
    """The matrix T of Eq. d3_transform (d x d, symmetric)."""
    lam = np.asarray(lam, dtype=np.float64)
    g, gp = g_and_gprime(lam, alpha, kind)
    lj = lam[:, None]
    ll = lam[None, :]
    diff = lj - ll
    scale = np.maximum(1.0, np.maximum(np.abs(lj), np.abs(ll)))
    near = np.abs(diff) <= NEAR_EQUAL * scale
    with np.errstate(divide="ignore", invalid="ignore"):
        T = (g[:, None] - g[None, :]) / diff
    _, gmid = g_and_gprime(0.5 * (lj + ll)[near], alpha, kind)
    T[near] = gmid
    return T
