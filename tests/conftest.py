import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a library)")
    config.addinivalue_line("markers", "slow: longer statistical runs")


@pytest.fixture(scope="session")
def orc_tables():
    """Oracle tables with the default parameters, built once and cached beside the oracle build."""
    import oracle

    oracle.build()
    path = os.path.join(ROOT, "oracle", "_build", "tables_default.npz")
    src = os.path.join(ROOT, "oracle", "qed_oracle.c")
    if os.path.exists(path) and os.path.getmtime(path) > os.path.getmtime(src):
        return oracle.Tables.load(path)
    t = oracle.Tables()
    tmp = path + f".{os.getpid()}.npz"
    t.save(tmp)
    os.replace(tmp, path)
    return t


@pytest.fixture(scope="session")
def golden():
    import json

    with open(os.path.join(ROOT, "tests", "golden", "paper_values.json")) as f:
        return json.load(f)
