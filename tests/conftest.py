import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: CPU test that takes more than ~10 s")


def to_oracle(p):
    """ModelParams (workloads) -> OracleParams: the same numbers, field by field."""
    import oracle
    names = oracle.OracleParams.__dataclass_fields__
    return oracle.OracleParams(**{k: getattr(p, k) for k in names})


def rel_err(a, b):
    """Relative error max|a - b| / max|b| (infinity norm)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (den if den > 0 else 1.0))


@pytest.fixture(scope="session")
def gpu_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False
