"""Shared fixtures.  GPU tests carry ``@pytest.mark.gpu``."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: larger workloads")


@pytest.fixture(scope="session")
def tiny_scene():
    import scenegen
    return scenegen.make_scene("tiny")


@pytest.fixture(scope="session")
def small_sh3_scene():
    """20k leaves with SH degree 3 in a 30x30x8 m box (several tiles deep)."""
    import scenegen
    leaves = scenegen.gen_leaves(20000, 7, kind="box", sh_degree=3,
                                 box=(0.0, 30.0, 0.0, 30.0, 0.0, 8.0), logscale=(-3.0, 0.5))
    sc = scenegen.build_tree(leaves)
    sc["config"] = "small_sh3"
    return sc


def rng(seed=0):
    return np.random.default_rng(seed)
