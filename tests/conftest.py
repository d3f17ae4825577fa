import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libxdg")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def dense_from_bsr(row_ptr, col, val):
    import numpy as np
    nb, Np = len(row_ptr) - 1, val.shape[-1]
    A = np.zeros((nb * Np, nb * Np))
    for i in range(nb):
        for z in range(row_ptr[i], row_ptr[i + 1]):
            j = col[z]
            A[i * Np:(i + 1) * Np, j * Np:(j + 1) * Np] = val[z]
    return A
