import os
import sys
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parent.parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the product kernels)")
    config.addinivalue_line("markers", "slow: long-running (full-size workloads)")


@pytest.fixture(scope="session")
def tiny_cfg():
    import synthlf
    return synthlf.CONFIGS["tiny"]


@pytest.fixture(scope="session")
def tiny_lf(tiny_cfg):
    import synthlf
    c = tiny_cfg
    return synthlf.make_lf(c.seed, c.nu, c.nv, c.width, c.height, c.n_planes, c.disp_max, c.texture)


@pytest.fixture(scope="session")
def ragged_lf():
    """Odd, non-square grid and image sizes that are not multiples of the
    block size: 1- and 2-member clusters and partial edge blocks."""
    import synthlf
    return synthlf.make_lf(11, 5, 3, 37, 29, 3, 4.0, "pink")


@pytest.fixture(scope="session")
def tiny_streams(tiny_lf, tiny_cfg):
    """Oracle streams of the tiny light field at q = 1 and the config's q."""
    import oracle
    c = tiny_cfg
    return {
        q: oracle.encode(tiny_lf, c.levels, c.block, c.search, q, debug=True)
        for q in (1, c.qstep)
    }
