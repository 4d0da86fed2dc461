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
    from oracle.model import GPModel, KernelSpec
    ks = [KernelSpec(kind=k["kind"], cols=tuple(k["cols"]), jitter=k["jitter"],
                     prior_a=tuple(k["prior_a"]), prior_b=tuple(k["prior_b"]))
          for k in problem["kernels"]]
    return GPModel(X=np.asarray(problem["X"], dtype=np.float64),
                   y=np.asarray(problem["y"], dtype=np.float64), kernels=ks,
                   lik=problem["lik"], noise_var=problem["noise_var"],
                   sample_hypers=problem["sample_hypers"], u_fixed=problem["u_fixed"])


@pytest.fixture
def oracle_model():
    return to_oracle_model
