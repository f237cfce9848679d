import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running (oracle at full size); still part of its marker set")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


def launches_per_role(pr: dict, role: str) -> list:
    """Launch counts of the kernels that do one job in a step, whichever implementation ran it."""
    names = {"density": ("ntilde", "tc_dens"), "force": ("force", "tc_force")}[role]
    return [pr[k][1] for k in names if k in pr]
