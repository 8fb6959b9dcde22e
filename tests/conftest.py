import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300)")
    config.addinivalue_line("markers", "slow: long-running statistical check")


@pytest.fixture(scope="session")
def pdf():
    from paper_2511_19633_gb300 import inputs
    return inputs.synthetic_pdf_grid()


@pytest.fixture(scope="session")
def oracle_mod():
    from oracle import oracle
    oracle.build()
    return oracle


def binomial_close(p_mc, p_true, n, nsig=4.5):
    sig = np.sqrt(max(p_true * (1.0 - p_true), 1e-12) / n)
    return abs(p_mc - p_true) <= nsig * sig + 1e-9
