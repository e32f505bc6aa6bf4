import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and runs the CUDA path")
    config.addinivalue_line("markers", "slow: full-size parity case")


@pytest.fixture(scope="session")
def orc():
    import oracle
    return oracle


@pytest.fixture(scope="session")
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1007_4400_gb300 import gevp
    gevp.load()
    return torch.device("cuda", 0)


def crandn(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)


def rand_hpd(rng, n, cond=10.0):
    Q, _ = np.linalg.qr(crandn(rng, n, n))
    d = np.exp(np.linspace(0, np.log(cond), n))
    B = (Q * d) @ Q.conj().T
    return 0.5 * (B + B.conj().T)


def rand_herm(rng, n):
    G = crandn(rng, n, n)
    return 0.5 * (G + G.conj().T)
