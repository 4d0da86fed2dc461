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
    """Workload dict -> oracle GPModel."""
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
