import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")
    # temporary files (the mutant oracles' builds) stay inside the repository,
    # one directory per session (a mutant's child session has its own),
    # removed when the session ends
    if not config.option.basetemp and not hasattr(config, "workerinput"):
        os.makedirs(os.path.join(ROOT, ".pytest_tmp"), exist_ok=True)
        config.option.basetemp = os.path.join(ROOT, ".pytest_tmp", f"session-{os.getpid()}")
        config._celeris_basetemp = config.option.basetemp


def pytest_unconfigure(config):
    path = getattr(config, "_celeris_basetemp", None)
    if path:
        shutil.rmtree(path, ignore_errors=True)


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.lib()
    return oracle
