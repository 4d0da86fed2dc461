"""Planted mistakes in the oracle, each caught by one of its pins (CPU only).

The oracle is trusted because its pins (finite differences, closed forms, library routines,
higher-precision evaluations, brute force) tie it to the mathematics rather than to itself. This
file checks that the pins are sharp enough: for each plausible mistake (a dropped term, a wrong
sign, a wrong index, a transposed operand, a wrong constant, an explicit step where the method is
implicit) it builds a copy of the oracle module with that one textual change, swaps the changed
function or class in for the length of one test, and requires a named pin to fail with an
assertion. The real oracle is never edited; the swap is undone when the test ends.
"""
import importlib
import inspect
import os
import sys
import types
from dataclasses import dataclass
from typing import Callable, Tuple

import pytest

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import test_oracle_bme as pins_bme  # noqa: E402
import test_oracle_geometry as pins_geo  # noqa: E402
import test_oracle_integrator as pins_int  # noqa: E402
import test_oracle_model as pins_model  # noqa: E402
import test_oracle_primal as pins_primal  # noqa: E402
import test_oracle_rng_jacobi as pins_rng  # noqa: E402


@dataclass
class Mistake:
    id: str
    module: str            # the oracle module the mistake is planted in
    old: str               # text that occurs exactly once in that module's source
    new: str               # what it becomes
    names: Tuple[str, ...]  # the functions / classes ("Class.method" for one method) swapped in
    pin: Callable          # pin(oracle_model) must raise AssertionError with the mistake planted


def mutant_module(module, old, new):
    """A fresh copy of `module` executed from its source with `old` replaced by `new`."""
    src = inspect.getsource(module)
    assert src.count(old) == 1, f"{module.__name__}: {old!r} occurs {src.count(old)} times"
    mod = types.ModuleType(module.__name__)
    mod.__package__ = module.__package__
    mod.__file__ = module.__file__
    exec(compile(src.replace(old, new), module.__file__, "exec"), mod.__dict__)
    return mod


def plant(monkeypatch, mistake):
    """Swap the mutant's objects in for the real ones wherever the real ones are referenced (the
    oracle's own modules and the pin modules that imported them by name)."""
    real = importlib.import_module(mistake.module)
    fake = mutant_module(real, mistake.old, mistake.new)
    for name in mistake.names:
        if "." in name:
            cls, attr = name.split(".")
            monkeypatch.setattr(getattr(real, cls), attr, getattr(getattr(fake, cls), attr))
            continue
        orig, repl = getattr(real, name), getattr(fake, name)
        for m in list(sys.modules.values()):
            d = getattr(m, "__dict__", None)
            if isinstance(d, dict) and d.get(name) is orig:
                monkeypatch.setattr(m, name, repl)


# ---- the dual GP model (oracle/model.py, oracle/kernels.py) -------------------------------------
MISTAKES = [
    Mistake("lik-third-derivative-sign", "oracle.model",
            "s * (1.0 - s) * (1.0 - 2.0 * s)", "s * (1.0 - s) * (2.0 * s - 1.0)",
            ("lik_derivs",), lambda om: pins_model.test_third_derivatives_fd(0, om)),
    Mistake("potential-drops-log-det-K", "oracle.model",
            "U += 0.5 * s.quad + 0.5 * s.logdet + 0.5 * model.N * LOG2PI",
            "U += 0.5 * s.quad + 0.5 * model.N * LOG2PI",
            ("potential",), lambda om: pins_model.test_potential_matches_scipy_densities(0, om)),
    Mistake("gradient-drops-trace-term", "oracle.model",
            "+ 0.5 * np.trace(s.Kinv @ Kh)", "+ 0.0",
            ("gradient",), lambda om: pins_model.test_gradient_fd(0, om)),
    Mistake("hessian-f-u-column-sign", "oracle.model",
            "col = -s.Kinv @ s.d(h) @ s.alpha", "col = s.Kinv @ s.d(h) @ s.alpha",
            ("hessian",), lambda om: pins_model.test_hessian_fd(0, om)),
    Mistake("hessian-drops-hyperprior-curvature", "oracle.model",
            "v += spec.prior_b[h] * np.exp(-u[k, h])", "v += 0.0",
            ("hessian",), lambda om: pins_model.test_hessian_fd(0, om)),
    Mistake("third-uuu-drops-a-trace", "oracle.model",
            "+ 0.5 * np.trace(Sk @ Sj @ Sl)", "",
            ("ThirdDerivatives",), lambda om: pins_model.test_third_derivatives_fd(0, om)),
    Mistake("third-ff-wrong-sample-index", "oracle.model",
            "D[a * N + m, b * N + m] += self.tau * self.l3[m]",
            "D[a * N + m, b * N + m] += self.tau * self.l3[(m + 1) % N]",
            ("ThirdDerivatives",), lambda om: pins_model.test_third_derivatives_fd(0, om)),
    Mistake("third-uff-sign", "oracle.model",
            "D[np.ix_(ik, ik)] = -self._A(k, jh)", "D[np.ix_(ik, ik)] = self._A(k, jh)",
            ("ThirdDerivatives",), lambda om: pins_model.test_third_derivatives_fd(0, om)),
    Mistake("se-third-kernel-derivative-coefficient", "oracle.kernels",
            "r ** 3 - 6.0 * r * r + 4.0 * r", "r ** 3 - 6.0 * r * r + 2.0 * r",
            ("kernel_derivs",), lambda om: pins_model.test_kernel_higher_derivatives_fd("se")),
    Mistake("overlap-second-kernel-derivative-sign", "oracle.kernels",
            "D2 = c * E * (s * s - s)", "D2 = c * E * (s * s + s)",
            ("kernel_derivs",), lambda om: pins_model.test_kernel_higher_derivatives_fd("overlap")),
]

# ---- SoftAbs map and Riemannian geometry (oracle/softabs.py, oracle/geometry.py) ----------------
MISTAKES += [
    Mistake("gprime-sign-of-second-term", "oracle.softabs",
            "gpm = 1.0 / th - xm / (sh * sh)", "gpm = 1.0 / th + xm / (sh * sh)",
            ("g_and_gprime",), lambda om: pins_geo.test_g_matches_mpmath(1e6)),
    Mistake("gprime-series-drops-cubic-term", "oracle.softabs",
            "gp[small] = 2.0 * xs / 3.0 - 4.0 * xs * x2 / 45.0 + 4.0 * xs * x2 * x2 / 315.0",
            "gp[small] = 2.0 * xs / 3.0 + 4.0 * xs * x2 * x2 / 315.0",
            ("g_and_gprime",), lambda om: pins_geo.test_g_matches_mpmath(1e6)),
    Mistake("divided-difference-absolute-denominator", "oracle.softabs",
            "T = (g[:, None] - g[None, :]) / diff", "T = (g[:, None] - g[None, :]) / np.abs(diff)",
            ("divided_differences",), lambda om: pins_geo.test_divided_differences_mpmath()),
    Mistake("W1-without-divided-differences", "oracle.geometry",
            "return self.Psi @ (np.outer(b, b) * self.T) @ self.Psi.T",
            "return self.Psi @ np.outer(b, b) @ self.Psi.T",
            ("Geometry.W1",), lambda om: pins_geo.test_betancourt_traces_match_fd_of_metric(3.0, "coth", om)),
    Mistake("W2-with-R-instead-of-R-o-T", "oracle.geometry",
            "return (self.Psi * (self.gp / self.g)) @ self.Psi.T",
            "return (self.Psi * (1.0 / self.g)) @ self.Psi.T",
            ("Geometry.W2",), lambda om: pins_geo.test_betancourt_traces_match_fd_of_metric(3.0, "coth", om)),
    Mistake("dHdq-as-printed", "oracle.geometry",
            "return self.dU + 0.5 * self.traces(self.W2()) - 0.5 * self.traces(self.W1(p))",
            "return self.dU - 0.5 * self.traces(self.W2()) + 0.5 * self.traces(self.W1(p))",
            ("Geometry.dHdq",), lambda om: pins_geo.test_dHdq_matches_fd_of_hamiltonian(1e6, "coth", om)),
    Mistake("Ginv-p-transposed-eigenvectors", "oracle.geometry",
            "return self.Psi @ ((self.Psi.T @ p) / self.g)",
            "return self.Psi.T @ ((self.Psi @ p) / self.g)",
            ("Geometry.Ginv_p",), lambda om: pins_geo.test_dHdq_matches_fd_of_hamiltonian(1e6, "coth", om)),
    Mistake("hamiltonian-drops-log-det-G", "oracle.geometry",
            "0.5 * (d * LOG2PI + self.logdetG())", "0.5 * (d * LOG2PI)",
            ("Geometry.hamiltonian",),
            lambda om: pins_geo.test_dHdq_matches_fd_of_hamiltonian(1e6, "coth", om)),
    Mistake("momentum-root-uses-g-not-sqrt-g", "oracle.geometry",
            "return self.Psi @ (np.sqrt(self.g) * (self.Psi.T @ z))",
            "return self.Psi @ (self.g * (self.Psi.T @ z))",
            ("Geometry.sqrtG_z",), lambda om: pins_geo.test_momentum_root_is_symmetric_square_root(om)),
]

# ---- integrator, sampler, generator, Jacobi, BME (oracle/integrator.py ... oracle/bme.py) -------
MISTAKES += [
    Mistake("leapfrog-explicit-momentum-half-step", "oracle.integrator",
            "ph = p - 0.5 * eps * geo.dHdq(ph)", "ph = p - 0.5 * eps * geo.dHdq(p)",
            ("leapfrog",), lambda om: pins_int.test_leapfrog_is_reversible(om)),
    Mistake("leapfrog-explicit-position-step", "oracle.integrator",
            "qn = q + 0.5 * eps * (v0 + gk.dHdp(ph))", "qn = q + eps * v0",
            ("leapfrog",), lambda om: pins_int.test_leapfrog_is_reversible(om)),
    Mistake("metropolis-hastings-inverted", "oracle.sampler",
            "logr < H0 - H1", "logr < H1 - H0",
            ("sample",), lambda om: pins_int.test_metropolis_hastings_keeps_the_posterior_at_a_coarse_step(om)),
    Mistake("philox-multiplier", "oracle.philox",
            "M0 = 0xD2E7470EE14C6C93", "M0 = 0xD2E7470EE14C6C95",
            ("philox4x64_10",),
            lambda om: pins_rng.test_philox_matches_numpy_library((7, 9), (5, 3, 2, 1))),
    Mistake("philox-round-swaps-products", "oracle.philox",
            "x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0",
            "x0, x1, x2, x3 = hi0 ^ x1 ^ k0, lo1, hi1 ^ x3 ^ k1, lo0",
            ("philox4x64_10",),
            lambda om: pins_rng.test_philox_matches_numpy_library((7, 9), (5, 3, 2, 1))),
    Mistake("box-muller-radius", "oracle.philox",
            "r = np.sqrt(-2.0 * np.log(u1))", "r = np.sqrt(-np.log(u1))",
            ("normals",), lambda om: pins_rng.test_box_muller_normals_are_standard()),
    Mistake("jacobi-rotation-sign", "oracle.jacobi",
            "M[:, j] = c * Mj - s * Ml", "M[:, j] = c * Mj + s * Ml",
            ("jacobi_eigh",), lambda om: pins_rng.test_jacobi_matches_eigh(5)),
    Mistake("bme-right-endpoint-rule", "oracle.bme",
            "est = float(np.sum(0.5 * (e[1:] + e[:-1]) * dt))", "est = float(np.sum(e[1:] * dt))",
            ("thermodynamic_integration",), lambda om: pins_bme.test_trapezoid_on_a_closed_form_integrand()),
    Mistake("bme-variance-weights", "oracle.bme",
            "w[1:] += 0.5 * dt", "w[1:] += dt",
            ("thermodynamic_integration",),
            lambda om: pins_bme.test_variance_formula_matches_replicated_estimates()),
]

# ---- the primal reduced-rank model and the mean/variance model (oracle/primal.py) ---------------
MISTAKES += [
    Mistake("primal-hessian-coefficient-prior", "oracle.primal",
            "H[i, i] += eh[m]", "H[i, i] += 0.5 * eh[m]",
            ("hessian",), lambda om: pins_primal.test_gradient_and_hessian_match_finite_differences("bernoulli")),
    Mistake("primal-third-drops-a-chain-rule-term", "oracle.primal",
            "hjk[j, j2] * hj[j3] + hjk[j, j3] * hj[j2] + hjk[j2, j3] * hj[j]",
            "hjk[j, j2] * hj[j3] + hjk[j, j3] * hj[j2]",
            ("ThirdDerivatives",),
            lambda om: pins_primal.test_third_derivatives_match_finite_differences("bernoulli")),
    Mistake("meanvar-third-derivative-drops-a-term", "oracle.primal",
            "dA = -rho * (1.0 - rho) + z * rho + 2.0", "dA = -rho * (1.0 - rho) + 2.0",
            ("data_derivs",), lambda om: pins_primal.test_meanvar_likelihood_derivatives_match_finite_differences()),
]

MISTAKES += [
    Mistake("primal-spectral-weight-exponent-as-printed", "oracle.primal",
            "np.exp(-pi * pi * m * m * s / (16.0 * model.L ** 2))",
            "np.exp(-pi * m * m * s / (16.0 * model.L ** 2))",
            ("spectral_weights",),
            lambda om: pins_primal.test_spectral_weights_are_the_fourier_transform_of_the_kernel(1.0)),
    Mistake("primal-feature-frequency", "oracle.primal",
            "(model.Xg[:, k:k + 1] + model.L) / (2.0 * model.L)", "(model.Xg[:, k:k + 1] + model.L) / model.L",
            ("features",), lambda om: pins_primal.test_reduced_rank_features_reproduce_the_kernel()),
    Mistake("tempered-mean-drops-posterior-variance", "oracle.bme",
            "- 0.5 * (r @ r + np.trace(Sig)) / noise_var", "- 0.5 * (r @ r) / noise_var",
            ("gaussian_tempered_loglik_mean",),
            lambda om: pins_bme.test_gaussian_gp_evidence_is_the_integral_of_the_tempered_means()),
    Mistake("jacobi-eigenvectors-not-rotated", "oracle.jacobi",
            "Psi[:, l] = s * Pj + c * Pl", "Psi[:, l] = Pl",
            ("jacobi_eigh",), lambda om: pins_rng.test_jacobi_matches_eigh(5)),
    Mistake("jacobi-warm-start-ignored", "oracle.jacobi",
            "Psi = np.eye(d) if Psi0 is None else np.array(Psi0, dtype=np.float64)", "Psi = np.eye(d)",
            ("jacobi_eigh",),
            lambda om: pins_rng.test_jacobi_warm_start_needs_one_to_two_sweeps_cold_grows_with_d()),
    Mistake("momentum-drawn-from-identity", "oracle.sampler",
            "p = geo.sqrtG_z(z)", "p = z",
            ("sample",), lambda om: pins_int.test_metropolis_hastings_keeps_the_posterior_at_a_coarse_step(om)),
    Mistake("log-det-G-from-absolute-eigenvalues", "oracle.geometry",
            "return float(np.sum(np.log(self.g)))", "return float(np.sum(np.log(np.abs(self.lam))))",
            ("Geometry.logdetG",),
            lambda om: pins_geo.test_betancourt_traces_match_fd_of_metric(3.0, "coth", om)),
]

MISTAKES += [
    Mistake("sampler-records-U-not-log-P", "oracle.sampler",
            "out_lp.append(-geo.U)", "out_lp.append(geo.U)",
            ("sample",), lambda om: pins_int.test_sampler_records_the_log_posterior_of_its_samples(om)),
    Mistake("linear-kernel-derivative-drops-amplitude", "oracle.kernels",
            "D1 = np.full((N, N), c * th)", "D1 = np.full((N, N), th)",
            ("kernel_derivs",), lambda om: pins_model.test_kernel_higher_derivatives_fd("linear")),
    Mistake("overlap-third-kernel-derivative-drops-a-term", "oracle.kernels",
            "D3 = c * E * (s ** 3 - 3.0 * s * s + s)", "D3 = c * E * (s ** 3 - 3.0 * s * s)",
            ("kernel_derivs",), lambda om: pins_model.test_kernel_higher_derivatives_fd("overlap")),
    Mistake("primal-potential-drops-bias-prior", "oracle.primal",
            "U += 0.5 * b * b / model.bias_var + 0.5 * log(model.bias_var)",
            "U += 0.5 * log(model.bias_var)",
            ("potential",), lambda om: pins_primal.test_potential_matches_scipy_densities("bernoulli")),
    Mistake("meanvar-cross-derivative-sign", "oracle.primal",
            "(0, 1): r * rho / v,", "(0, 1): -r * rho / v,",
            ("data_derivs",), lambda om: pins_primal.test_meanvar_likelihood_derivatives_match_finite_differences()),
    Mistake("philox-weyl-increment", "oracle.philox",
            "W0 = 0x9E3779B97F4A7C15", "W0 = 0x9E3779B97F4A7C17",
            ("philox4x64_10",),
            lambda om: pins_rng.test_philox_matches_numpy_library((7, 9), (5, 3, 2, 1))),
]


@pytest.mark.parametrize("mistake", MISTAKES, ids=[m.id for m in MISTAKES])
def test_planted_mistake_fails_its_pin(mistake, monkeypatch, oracle_model):
    plant(monkeypatch, mistake)
    with pytest.raises(AssertionError):
        mistake.pin(oracle_model)


@pytest.mark.parametrize("mistake", [m for m in MISTAKES if m.id in (
    "gradient-drops-trace-term", "third-uuu-drops-a-trace", "dHdq-as-printed", "leapfrog-explicit-position-step",
    "philox-multiplier", "primal-third-drops-a-chain-rule-term")], ids=lambda m: m.id)
def test_the_swap_itself_changes_nothing(mistake, monkeypatch, oracle_model):
    """Control: the same swap with the text left unchanged keeps the pin passing, so a failure
    above comes from the planted mistake, not from running a copy of the module."""
    plant(monkeypatch, Mistake(mistake.id, mistake.module, mistake.old, mistake.old, mistake.names,
                               mistake.pin))
    mistake.pin(oracle_model)
