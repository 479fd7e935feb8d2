import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")


_WL = {}


@pytest.fixture(scope="session")
def workload():
    from paper_2605_21398_gb300 import synth

    def get(name, **kw):
        key = (name, tuple(sorted(kw.items())))
        if key not in _WL:
            _WL[key] = synth.make_workload(name, **kw)
        return _WL[key]
    return get
