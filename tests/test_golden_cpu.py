"""Checks against values the paper prints (fixtures under tests/golden/, each line with its
citation): the simulated logistic-regression recipe and model dimensions of Sec. 2.5 / Fig. 1,
the integrator settings of those runs, and the 101-point inverse-temperature schedule, which the
oracle's trapezoid rule then integrates to within its error bound (CPU only)."""
import inspect
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle import primal  # noqa: E402
from oracle.bme import thermodynamic_integration  # noqa: E402
from paper_2511_06407_b300 import bme, rmhmc, workloads as wl  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    """Non-comment lines of a fixture as lists of whitespace-separated fields (citation dropped)."""
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                out.append(line.split("|", 1)[0].split())
    return out


def _settings():
    rows = _rows("simulated_logistic_sec2_5.txt")
    one = {r[0]: [float(v) for v in r[1:]] for r in rows if r[0] != "d_of_D"}
    dims = [(int(r[1]), int(r[2])) for r in rows if r[0] == "d_of_D"]
    return one, dims


def test_simulated_logistic_recipe_matches_the_printed_values():
    g, _ = _settings()
    defaults = {k: v.default for k, v in inspect.signature(wl.solin_logistic).parameters.items()}
    assert defaults["N"] == int(g["N"][0]) and defaults["M"] == int(g["M"][0])
    assert defaults["L"] == g["L"][0] and defaults["bias"] == g["b_star"][0]
    assert defaults["sd"] == g["sd_f_star"][0]
    prob = wl.solin_logistic(1, seed=0)
    f = prob["f_true"]
    assert len(f) == int(g["N"][0]) and abs(f.std() - g["sd_f_star"][0]) < 1e-12
    # the truth lies in the span of the features with 4 <= m <= 16 and a constant, and not in the
    # span of the others (the low-frequency sines are nearly collinear with the constant on the
    # data's range, so the coefficients themselves are not identifiable: test the residuals)
    M, L = prob["M"], prob["L"]
    m = np.arange(1, M + 1)
    x = prob["Xg"][:, 0]
    feats = np.sin(np.pi * m[None, :] * (x[:, None] + L) / (2 * L))
    lo, hi = (int(v) for v in g["m_nonzero"])
    active = (m >= lo) & (m <= hi)

    def residual(cols):
        A = np.column_stack([feats[:, cols], np.ones_like(x)])
        c, *_ = np.linalg.lstsq(A, f, rcond=None)
        return np.linalg.norm(A @ c - f) / np.linalg.norm(f)

    assert residual(active) < 1e-10
    assert residual(m < lo) > 1e-2
    assert set(np.unique(prob["y"])) <= {0.0, 1.0}


def test_model_dimension_follows_the_printed_pairs():
    _, dims = _settings()
    assert dims == [(1, 34), (16, 484)]
    for D, d in dims:
        prob = wl.solin_logistic(D, N=20, seed=0)
        assert primal.from_problem(prob).d == d == wl.dims(prob)[2]


def test_benchmark_uses_the_printed_integrator_settings():
    g, _ = _settings()
    assert bench.SOLIN_EPS == g["eps"][0]
    assert bench.SOLIN_KAPPA == g["kappa"][0]
    assert rmhmc.Integrator().jacobi_tol == g["zeta"][0]


def test_piecewise_schedule_matches_the_printed_pieces():
    tau = bme.piecewise_schedule()
    assert tau.shape == (101,)
    covered = 0
    for s_lo, s_hi, start, step, s0 in _rows("temperature_schedule_sec2_5.txt"):
        s = np.arange(int(s_lo), int(s_hi) + 1)
        want = float(start) - float(step) * (s - int(s0))
        np.testing.assert_allclose(tau[s - 1], want, rtol=0, atol=1e-15)
        covered += len(s)
    assert covered == 101
    assert tau[0] == 1.0 and abs(tau[-1]) < 1e-15
    assert np.all(np.diff(tau) < 0)
    # the pieces join: each piece's formula at its s0 gives the previous piece's last value
    np.testing.assert_allclose(tau[[40, 70, 90]], [0.2, 0.05, 0.01], rtol=0, atol=1e-15)


def test_oracle_trapezoid_over_the_printed_schedule_is_within_its_bound():
    """int_0^1 exp(-3 tau) d tau = (1 - e^-3) / 3; the trapezoid rule on any grid overestimates a
    convex integrand by at most sum_i h_i^3 max|f''| / 12 with max|f''| = 9."""
    tau = bme.piecewise_schedule()
    est, _ = thermodynamic_integration(tau, np.exp(-3.0 * tau))
    exact = (1.0 - math.exp(-3.0)) / 3.0
    h = np.abs(np.diff(tau))
    assert 0.0 < est - exact <= np.sum(h ** 3) * 9.0 / 12.0
