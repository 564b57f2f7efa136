import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

np.seterr(invalid="ignore", divide="ignore")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def _ensure_ucgen():
    from paper_2512_06715_gb300 import build
    build.build_ucgen()


@pytest.fixture(scope="session", autouse=True)
def _built_generator():
    _ensure_ucgen()


def instance_lp(inst):
    from oracle.lp import lp_from_arrays
    return lp_from_arrays(inst.row_ptr, inst.col, inst.val, inst.q, inst.c, inst.l, inst.u, inst.m_eq)


@pytest.fixture(scope="session")
def tiny24():
    """24-bus, 33-generator, 24-period instance (seed 0) and its LP."""
    from paper_2512_06715_gb300.instances import workload
    inst = workload("uc24_g33_T24")
    return inst, instance_lp(inst)


@pytest.fixture(scope="session")
def tiny24_oracle(tiny24):
    """FP64 oracle PDHG solution of the 24-bus instance to rel-KKT 1e-8."""
    from oracle.pdhg import pdhg_solve
    _, lp = tiny24
    res = pdhg_solve(lp, tol=1e-8, max_attempts=2_000_000)
    assert res.status == "optimal"
    return res
