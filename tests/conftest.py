import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a); runs the CUDA path through the C-ABI")
    config.addinivalue_line("markers", "slow: long-running; still part of its marker's suite")
    config.addinivalue_line("markers", "oracle_fullsize(scales): compares with the oracle run on the whole graph "
                                       "of these scales (started in child processes when the session begins)")


ORACLE_SEED = 1


def pytest_collection_finish(session):
    """Start the whole-graph oracle runs that the selected tests need, in
    child processes, so that they overlap the GPU tests collected before them."""
    scales = set()
    for item in session.items:
        m = item.get_closest_marker("oracle_fullsize")
        if m and m.args:
            scales.update(m.args[0])
    runs = {}
    if scales:
        from oracle import fullsize

        runs = {s: fullsize.start(s, ORACLE_SEED) for s in sorted(scales)}
    session.config.pp_oracle_runs = runs


def pytest_sessionfinish(session, exitstatus):
    for run in getattr(session.config, "pp_oracle_runs", {}).values():
        run.cancel()


@pytest.fixture(scope="session", autouse=True)
def built_libraries():
    """Build (or confirm up to date) the input generator, the oracle and libpp."""
    import kernel0.build
    import oracle.build
    import paper_1603_01876_gb300.build

    kernel0.build.build()
    oracle.build.build()
    paper_1603_01876_gb300.build.build()


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle

    return oracle


@pytest.fixture(scope="session")
def k0():
    import kernel0

    kernel0.lib()
    return kernel0
