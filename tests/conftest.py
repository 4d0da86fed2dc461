import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU check")


def to_oracle_model(problem):
    """Workload dict -> oracle model (GPModel, or PrimalModel for the reduced-rank model)."""
    if problem.get("model") == "primal":
        from oracle.primal import from_problem as primal_from_problem
        return primal_from_problem(problem)
    from oracle.model import from_problem
    return from_problem(problem)


@pytest.fixture
def oracle_model():
    return to_oracle_model


def potential_rounding_bound(m, q):
    """First-order change of U when every entry of every K_k is perturbed by one unit roundoff
    (|dK_ij| <= u |K_ij|): u * sum_k [ |alpha_k|^T |K_k| |alpha_k| / 2 + sum_ij |K_k^-1|_ij |K_k|_ij / 2 ].
    Forming K in FP64 already commits this error, so no FP64 evaluation of U can beat it."""
    from oracle import model as mdl
    f, u = mdl.split(m, q)
    b = 0.0
    for k, spec in enumerate(m.kernels):
        st = mdl.KernelState(spec, m.X[:, list(spec.cols)], f[k], u[k])
        K = np.abs(st.mats[0])
        a = np.abs(st.alpha)
        b += 0.5 * a @ K @ a + 0.5 * np.sum(np.abs(st.Kinv) * K)
    return 2.0 ** -53 * b


def eigen_backward_bound(H, G, Ginv_p, sweeps, unit=2.0 ** -53):
    """First-order change of G^-1 p under a symmetric perturbation E of H with
    ||E|| <= 4u ||H||_2 per Jacobi sweep (the normwise backward error the rotations of Sec. 2.4
    commit): g(H + E) - g(H) = Psi (T o Psi^T E Psi) Psi^T (Daleckii-Krein) with |T_jl| <= 1 for
    both soft-abs maps, so G^-1 p moves by at most ||G^-1||_2 * 4u sweeps ||H||_2 * ||G^-1 p||."""
    ev = np.linalg.eigvalsh(G)
    h2 = float(np.abs(np.linalg.eigvalsh(H)).max())
    return (1.0 / ev.min()) * 4.0 * unit * max(int(sweeps), 1) * h2 * float(np.linalg.norm(Ginv_p))
