import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def oracle_mod():
    """The oracle package; CTQR_ORACLE_PKG names another copy of it (the
    mutation tests run the pins against deliberately broken copies)."""
    alt = os.environ.get("CTQR_ORACLE_PKG")
    if alt:
        import importlib.util
        spec = importlib.util.spec_from_file_location("oracle", os.path.join(alt, "__init__.py"),
                                                      submodule_search_locations=[alt])
        mod = importlib.util.module_from_spec(spec)
        sys.modules["oracle"] = mod
        spec.loader.exec_module(mod)
        mod.lib()
        return mod
    import oracle
    oracle.lib()
    return oracle
