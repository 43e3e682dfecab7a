import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
for p in (ROOT, os.path.join(ROOT, "oracle")):
    if p not in sys.path:
        sys.path.insert(0, p)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the compiled library")
    config.addinivalue_line("markers", "slow: long-running CPU oracle case")


@pytest.fixture(scope="session")
def params():
    import oracle as O
    return O.load_params()


@pytest.fixture(scope="session")
def golden():
    with open(os.path.join(ROOT, "tests", "golden", "paper_tables.json")) as fh:
        return json.load(fh)


@pytest.fixture(scope="session")
def toy_oracle(params):
    import oracle as O
    o = O.Oracle(params[0]["toy"])
    o.keygen(7)
    return o


@pytest.fixture(scope="session")
def toybts_oracle(params):
    import oracle as O
    o = O.Oracle(params[0]["toybts"])
    o.keygen(7)
    return o
