import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
TESTS = os.path.dirname(os.path.abspath(__file__))
if TESTS not in sys.path:
    sys.path.insert(0, TESTS)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.hookimpl(trylast=True)
def pytest_collection_modifyitems(session, config, items):
    # the large oracle runs take minutes: when a selected test compares with
    # them, start them all in worker processes now, so that they run while
    # the earlier tests run (after -m/-k deselection; not for --collect-only)
    if config.option.collectonly:
        return
    if any("oracle_pool" in getattr(it, "fixturenames", ()) for it in items):
        import _oracle_pool
        _oracle_pool.start()


@pytest.fixture(scope="session")
def oracle_pool():
    import _oracle_pool
    _oracle_pool.start()
    yield _oracle_pool
    _oracle_pool.shutdown()
