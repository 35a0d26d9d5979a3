import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def box_room():
    """Plain tiny workload: box room, 4 keyframes, 512-point scans, 1,024 particles."""
    import synth
    return synth.box_room_workload(seed=0)


@pytest.fixture(scope="session")
def box_room_tables(box_room):
    """FP64 oracle tables of the box-room keyframes (sigma 0.2 m, r_t 1.0 m)."""
    import oracle
    return [oracle.build_table(kf["points"], kf["grid"], 0.2, 1.0) for kf in box_room["keyframes"]]
